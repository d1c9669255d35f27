"""Shared test helpers (parameter builders); no method arithmetic."""
import dataclasses

import workloads

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)
QE = 1.602176634e-19
ME = 9.1093837015e-31


def vacuum(nx, ny, nz, dx, dy, dz, solver=0, courant=1.0, mur_order=2, space_charge=1,
           lambda_diag=1.0, gamma=1.0, **kw):
    """A run without undulator and without particles (rest frame == lab when gamma == 1)."""
    base = workloads.WORKLOADS["undulator_24x24x96"]
    return dataclasses.replace(
        base, name="vacuum", nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, solver=solver,
        courant=courant, mur_order=mur_order, space_charge=space_charge, und_kind=-1,
        K=0.0, lambda_u=lambda_diag, n_periods=0.0, dist_head=0.0, gamma=gamma, sig_z=0.0,
        n_particles=0, plane_dist=0.0, **kw)
