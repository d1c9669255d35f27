"""Seeded synthetic inputs shared by the CUDA library tests, the bench and the oracle.

This module holds input *data* only: lab-frame macro-particle arrays drawn from a
seeded generator, and the plain numbers that define each workload (grid sizes,
lab-frame mesh resolution, undulator and bunch parameters).  It performs none of
the method's arithmetic: no Lorentz boost, no field evaluation, no push, no
deposition.  Both the oracle and the CUDA library receive the same lab-frame
particle array (x, y, z, ux, uy, uz per particle; metres and gamma*beta) and boost
it themselves.

Bunch recipe (MITHRA manual, Sec. "Electron Bunch Generation", Eqs. uniform1D,
gaussian1D, gaussian2D, bunchingFactor, negativeExponential):
  * transverse positions and momenta: independent Gaussians (numpy PCG64);
  * longitudinal: Gaussian positions, either random ("random"), or a quiet start
    (evenly spaced quantiles of the Gaussian, "quiet") on which shot noise is laid;
  * energy: gamma*(1 + N(0, sigma_gamma/gamma)), u_z from gamma and u_perp;
  * bunching b at the lab resonant wavelength lambda_r: z -> z - (2 b / k_r) sin(k_r z + phase),
    which gives |<exp(j k_r z)>| = b to first order in b;
  * shot noise: slices of length lambda_r, per slice amplitude sqrt(-2 ln x_j)/sqrt(N_e,j)
    and a uniform phase on [0, 2 pi), applied with the same modulation.
Positions are relative to the bunch reference point (the bunch centre).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = ["Workload", "lab_bunch", "WORKLOADS", "serving_requests", "scaled"]


@dataclasses.dataclass
class Workload:
    """One run: mesh (lab frame), undulator, bunch and step count.

    Lengths are metres in the laboratory frame, as in the manual's job files
    ("all the parameters in job file are given in the laboratory frame").
    """

    name: str
    nx: int
    ny: int
    nz: int
    dx: float            # lab transverse resolution (equal in both frames)
    dy: float
    dz: float            # lab longitudinal resolution (the rest frame uses gamma0 * dz)
    solver: int          # 0 NSFD, 1 FD
    courant: float       # FD: fraction of the CFL bound
    mur_order: int
    space_charge: int
    substeps: int
    und_kind: int        # 0 planar, 1 helical, 2 optical plane wave, 3 optical Gaussian beam,
                         # 4 static undulator array, -1 none
    K: float             # undulator parameter K, or a0 for an optical undulator
    lambda_u: float      # undulator period, or laser wavelength
    n_periods: float
    pol_deg: float
    waist: float
    pulse_fwhm: float    # c*tau (intensity FWHM), lab length
    signal: int          # 0 Gaussian envelope, 1 flat-top (Gaussian rise, then constant)
    dist_head: float     # lab distance between undulator entrance and bunch head
    gamma: float
    rel_espread: float
    sig_x: float
    sig_y: float
    sig_z: float
    sig_ux: float
    sig_uy: float
    charge_e: float      # electrons in the bunch
    n_particles: int
    bunching: float
    lambda_r: float      # lab wavelength at which bunching / shot noise are laid
    shot_noise: int
    quiet: int
    plane_dist: float    # lab distance of the power plane ahead of the bunch centre
    norm_freq: float
    steps: int
    seed: int
    precision: int = 0   # 0 FP64 plain, 1 FP32-mixed
    gap: float = 0.0     # undulator array: lab gap between modules
    n_modules: int = 1   # undulator array: number of modules of n_periods each
    taper: float = 0.0   # undulator array: K_i = K + i * taper
    nf_min: float = 0.0  # radiated-power spectrum: normalised frequencies nf_min .. nf_max
    nf_max: float = 0.0
    nf_points: int = 0   # number of spectrum frequencies (0: no spectrum)
    bunch_every: int = 0 # bunch sampling every this many steps (0: off)
    seed_type: int = -1  # seed through TF/SF planes: -1 none, 0 plane wave, 1 Gaussian beam (+z)
    seed_a0: float = 0.0
    seed_lambda: float = 1.0
    seed_pol_deg: float = 0.0
    seed_waist: float = 0.0
    seed_focus: float = 0.0      # lab position of the seed's reference point / focus
    seed_offset: float = 0.0     # c t0
    seed_pulse_fwhm: float = 0.0 # c tau; <= 0: continuous
    seed_cep_deg: float = 0.0
    uniform: int = 0     # longitudinal profile: 0 Gaussian (rms sig_z), 1 uniform over [-sig_z, sig_z]
    optimize: int = 0    # optimize-bunch-position (Sec. MESH): mesh and power plane follow the bunch's
                         # drift before the undulator entrance, so it sits at its placed position inside


def lab_bunch(w: Workload, n: Optional[int] = None, seed: Optional[int] = None) -> np.ndarray:
    """Return an (n, 6) float64 array of lab-frame macro-particles for workload ``w``."""
    n = w.n_particles if n is None else int(n)
    rng = np.random.Generator(np.random.PCG64(w.seed if seed is None else seed))
    out = np.empty((n, 6), dtype=np.float64)
    out[:, 0] = rng.standard_normal(n) * w.sig_x
    out[:, 1] = rng.standard_normal(n) * w.sig_y
    if w.uniform:
        # uniform current over [-sig_z, sig_z] (sig_z is half the bunch length, Sec. BUNCH)
        if w.quiet:
            z = w.sig_z * (2.0 * (np.arange(n, dtype=np.float64) + 0.5) / n - 1.0)
            z = z[rng.permutation(n)]
        else:
            z = rng.uniform(-w.sig_z, w.sig_z, n)
    elif w.quiet:
        # evenly spaced quantiles of the Gaussian current profile (quiet start)
        from scipy.special import erfinv
        q = (np.arange(n, dtype=np.float64) + 0.5) / n
        z = w.sig_z * math.sqrt(2.0) * erfinv(2.0 * q - 1.0)
        z = z[rng.permutation(n)]
    else:
        z = rng.standard_normal(n) * w.sig_z
    ux = rng.standard_normal(n) * w.sig_ux
    uy = rng.standard_normal(n) * w.sig_uy
    g = w.gamma * (1.0 + w.rel_espread * rng.standard_normal(n))
    uz = np.sqrt(np.maximum(g * g - 1.0 - ux * ux - uy * uy, 0.0))
    if w.lambda_r > 0.0 and (w.bunching > 0.0 or w.shot_noise):
        kr = 2.0 * math.pi / w.lambda_r
        if w.bunching > 0.0:
            z = z - (2.0 * w.bunching / kr) * np.sin(kr * z)
        if w.shot_noise:
            sl = np.floor(z / w.lambda_r).astype(np.int64)
            lo = sl.min()
            counts = np.bincount(sl - lo)
            nslice = counts.size
            xj = 1.0 - rng.random(nslice)          # in (0, 1]
            phj = 2.0 * math.pi * rng.random(nslice)
            ne = np.maximum(counts * (w.charge_e / n), 1.0)
            bj = np.sqrt(-2.0 * np.log(xj)) / np.sqrt(ne)
            z = z - (2.0 * bj[sl - lo] / kr) * np.sin(kr * z + phj[sl - lo])
    out[:, 2] = z
    out[:, 3] = ux
    out[:, 4] = uy
    out[:, 5] = uz
    return out


def _w(**kw) -> Workload:
    base = dict(solver=0, courant=1.0, mur_order=2, space_charge=1, substeps=1,
                pol_deg=0.0, waist=0.0, pulse_fwhm=0.0, signal=0, bunching=0.0,
                lambda_r=0.0, shot_noise=0, quiet=0, norm_freq=1.0, sig_ux=0.0, sig_uy=0.0)
    base.update(kw)
    return Workload(**base)


# Mesh numbers below were sized once from the textbook FEL resonance so that a
# rest-frame period holds the stated number of cells; they are plain inputs here.
WORKLOADS = {
    # Plain FP64 undulator radiation, small: 24x24x96, 8192 particles, FD at Courant 0.9.
    "undulator_24x24x96": _w(
        name="undulator_24x24x96", nx=24, ny=24, nz=96,
        dx=1.150357e-4, dy=1.150357e-4, dz=4.696314e-6,
        solver=1, courant=0.9, mur_order=2, space_charge=1,
        und_kind=0, K=1.0, lambda_u=0.03, n_periods=10, dist_head=0.06,
        gamma=20.0, rel_espread=1e-3, sig_x=50e-6, sig_y=50e-6, sig_z=20e-6,
        charge_e=10e-12 / 1.602176634e-19, n_particles=8192,
        plane_dist=0.35 * 96 * 4.696314e-6, steps=300, seed=1235, precision=0),
    # FEL-like single run: 128x128x512, 2M particles, shot-noise phases, NSFD.
    "fel_128x128x512": _w(
        name="fel_128x128x512", nx=128, ny=128, nz=512,
        dx=1.055448e-5, dy=1.055448e-5, dz=9.900980e-8,
        und_kind=0, K=1.4, lambda_u=0.018, n_periods=50, dist_head=0.036,
        gamma=100.0, rel_espread=1e-4, sig_x=50e-6, sig_y=50e-6, sig_z=7e-6,
        sig_ux=0.02, sig_uy=0.02,
        charge_e=100e-12 / 1.602176634e-19, n_particles=2_000_000,
        lambda_r=1.782e-6, shot_noise=1, quiet=1,
        plane_dist=0.45 * 512 * 9.900980e-8, optimize=1, steps=2000, seed=1236, precision=1),
    # The FEL run through an undulator line: four 12-period modules two periods apart, the
    # undulator parameter tapered by -0.005 per module (Sec. UNDULATOR, static-undulator-array).
    "fel_array_128x128x512": _w(
        name="fel_array_128x128x512", nx=128, ny=128, nz=512,
        dx=1.055448e-5, dy=1.055448e-5, dz=9.900980e-8,
        und_kind=4, K=1.4, lambda_u=0.018, n_periods=12, dist_head=0.036,
        gap=0.036, n_modules=4, taper=-0.005,
        gamma=100.0, rel_espread=1e-4, sig_x=50e-6, sig_y=50e-6, sig_z=7e-6,
        sig_ux=0.02, sig_uy=0.02,
        charge_e=100e-12 / 1.602176634e-19, n_particles=2_000_000,
        lambda_r=1.782e-6, shot_noise=1, quiet=1,
        plane_dist=0.45 * 512 * 9.900980e-8, optimize=1, steps=2000, seed=1240, precision=1),
    # Seeded UV FEL (Example 2 job file): 2500 x 2500 x 165 um at 30 x 30 x 0.02 um, 4 194 304
    # particles of a uniform 150 um bunch (55 pC, gamma 391.36, 1e-4 energy spread), planar
    # undulator K = 1.95, 2.8 cm; a 10 kW Gaussian seed at 0.265187 um (a0 = 9.857e-7, waist
    # 183.74 um, focus 0.7 m), continuous.
    "seeded_uv_84x84x8250": _w(
        name="seeded_uv_84x84x8250", nx=84, ny=84, nz=8250,
        dx=30e-6, dy=30e-6, dz=0.02e-6, space_charge=0,
        und_kind=0, K=1.95, lambda_u=0.028, n_periods=536, dist_head=0.056,
        gamma=391.36, rel_espread=1e-4, sig_x=95.3e-6, sig_y=95.3e-6, sig_z=75.0e-6, uniform=1,
        sig_ux=0.0105, sig_uy=0.0105, quiet=1,
        charge_e=3.4332e8, n_particles=4_194_304,
        seed_type=1, seed_a0=9.857e-7, seed_lambda=0.265187e-6, seed_waist=183.74e-6,
        seed_focus=0.7, seed_offset=0.7, seed_pulse_fwhm=0.0,
        plane_dist=78e-6, steps=200, seed=1241, precision=1),
    # Large single run: 256x256x1024, 32M particles, helical undulator, 1% bunching.
    "helical_256x256x1024": _w(
        name="helical_256x256x1024", nx=256, ny=256, nz=1024,
        dx=3.314646e-6, dy=3.314646e-6, dz=1.562539e-8,
        und_kind=1, K=1.0, lambda_u=0.01, n_periods=125, dist_head=0.02,
        gamma=200.0, rel_espread=1e-4, sig_x=40e-6, sig_y=40e-6, sig_z=2.0e-6,
        sig_ux=0.02, sig_uy=0.02,
        charge_e=100e-12 / 1.602176634e-19, n_particles=32_000_000,
        bunching=0.01, lambda_r=2.5e-7, quiet=1,
        plane_dist=0.45 * 1024 * 1.562539e-8, optimize=1, steps=4000, seed=1237, precision=1),
    # Optical undulator (inverse Compton): 192x192x768, 4M particles, Gaussian laser.
    "ics_192x192x768": _w(
        name="ics_192x192x768", nx=192, ny=192, nz=768,
        dx=5.524703e-10, dy=5.524703e-10, dz=6.510925e-12,
        und_kind=3, K=0.5, lambda_u=1e-6, n_periods=0, waist=20e-6,
        pulse_fwhm=299792458.0 * 10e-12, signal=0, dist_head=0.0,
        gamma=60.0, rel_espread=1e-4, sig_x=2e-6, sig_y=2e-6, sig_z=3e-6,
        charge_e=100e-12 / 1.602176634e-19, n_particles=4_000_000,
        plane_dist=0.3 * 768 * 6.510925e-12, steps=6000, seed=1239, precision=1),
}


def scaled(w: Workload, **changes) -> Workload:
    """A copy of ``w`` with fields replaced (smaller grids / fewer particles for tests)."""
    return dataclasses.replace(w, **changes)


SERVING_GRIDS = ((32, 32, 128), (64, 64, 256), (96, 96, 384), (128, 128, 512))


def serving_requests(n_requests: int = 64, rate_hz: float = 4.0, seed: int = 1238,
                     steps_range=(500, 2000), np_range=(1e4, 1e6), grids=SERVING_GRIDS):
    """The serving stream: Poisson arrivals, random grid, particles, undulator, precision.

    Returns a list of (arrival_time_s, Workload).  Mesh resolution is sized from the
    textbook lab resonance lambda_u (1 + K^2/2) / (2 gamma^2): 12 cells per lab
    resonant wavelength along z, and a transverse cell of 1.5 rest-frame cells.  The bunch
    (rms length 0.08 of the mesh, head at 0.24) sits at the mesh centre once inside the
    undulator (optimize-bunch-position), and the power plane lies 0.38 of the mesh ahead of
    the centre: ahead of the head and 0.12 of the mesh inside the boundary.  `grids` replaces
    the four grid sizes (the draw picks one of them uniformly).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        nx, ny, nz = grids[int(rng.integers(0, len(SERVING_GRIDS)))  % len(grids)]
        npart = int(round(math.exp(rng.uniform(math.log(np_range[0]), math.log(np_range[1])))))
        npart = max(4, npart - npart % 4)
        gamma = float(rng.uniform(20.0, 150.0))
        K = float(rng.uniform(0.5, 2.0))
        lu = float(rng.uniform(0.01, 0.03))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        prec = int(rng.integers(0, 2))
        lam_r = lu * (1.0 + 0.5 * K * K) / (2.0 * gamma * gamma)
        dz = lam_r / 12.0
        g_und = gamma / math.sqrt(1.0 + 0.5 * K * K)
        dxy = 1.5 * g_und * dz
        w = _w(name=f"serve_{r}", nx=nx, ny=ny, nz=nz, dx=dxy, dy=dxy, dz=dz,
               und_kind=0, K=K, lambda_u=lu, n_periods=12, dist_head=2 * lu,
               gamma=gamma, rel_espread=1e-4, sig_x=0.15 * nx * dxy / 6.0,
               sig_y=0.15 * ny * dxy / 6.0, sig_z=0.08 * nz * dz,
               sig_ux=0.0, sig_uy=0.0, charge_e=50e-12 / 1.602176634e-19,
               n_particles=npart, plane_dist=0.38 * nz * dz, optimize=1, steps=steps,
               seed=seed * 1000 + r, precision=prec)
        out.append((t, w))
    return out
