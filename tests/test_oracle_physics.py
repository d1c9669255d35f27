"""Physics pins of the whole oracle step against closed forms.

* single electron in a planar undulator: transverse amplitude K/(gamma k_u), constant
  lab energy, zero mean rest-frame drift (the rest frame of Sec. "Lorentz Transformation");
* on-axis spectrum: the rest-frame field at the sampling plane peaks at w* = gamma0 beta0 c k_u,
  i.e. at the lab resonance lambda_u (1 + K^2/2) / (2 gamma^2) after the Doppler factor (helical:
  1 + K^2); an optical undulator gives the inverse-Compton lambda_L (1 + a0^2/2) / (4 gamma^2);
* optimize-bunch-position: the mesh shift equals the drift of the reference before it enters;
* initial bunching factor of a bunch modulated at the resonance equals the modulation;
* radiated-power diagnostic: cycle-averaged flux a^2/(2 mu0 c) of a plane wave, the Doppler
  factor gamma0^2 (1 + beta0)^2 to the lab, and coherent N^2 scaling;
* absolute radiated power: one electron in a weak undulator is, in the rest frame, a harmonic
  dipole, and the power through the sampling plane equals the dipole's flux through it;
* source signs and factors (Eqs. WaveA, WaveF): the potential around an electron is negative
  and a slowly moving charge has A_z / phi = v_z / c^2.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.helpers import C0, EPS0, MU0, QE, ME, vacuum


def _single_electron(gamma=20.0, K=1.0, lu=0.03, steps=440, substeps=1, optimize=0):
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, n_particles=1, charge_e=1.0, gamma=gamma, K=K, lambda_u=lu,
                         space_charge=0, substeps=substeps, optimize=optimize)
    lab = np.array([[0.0, 0.0, 0.0, 0.0, 0.0, math.sqrt(gamma * gamma - 1)]])
    r = oracle.Run(oracle.params_from(w), lab)
    traj = []
    for _ in range(steps):
        r.step(1)
        traj.append(r.particles()[0].copy())
    return r, w, np.array(traj)


def test_single_electron_undulator_trajectory():
    gamma, K, lu = 20.0, 1.0, 0.03
    r, w, tr = _single_electron(gamma, K, lu)
    inf = r.info()
    g0, b0, dt = inf["gamma0"], inf["beta0"], inf["dt"]
    ku = 2 * math.pi / lu
    u = tr[:, 3:]
    g = np.sqrt(1 + np.sum(u * u, axis=1))
    glab = g0 * (g + b0 * u[:, 2])
    # rest-frame time of each sample and the lab coordinate of the particle
    n = np.arange(len(tr)) + 1
    t = inf["T0"] + (n + 0.5) * dt
    zeta = g0 * (tr[:, 2] + b0 * C0 * t)
    inside = (zeta > 2 * lu) & (zeta < (w.n_periods - 1) * lu)
    assert inside.sum() > 150
    # lab energy is constant in a static magnetic field up to the O(dt^2) error of the scheme
    err1 = np.max(np.abs(glab[inside] - gamma)) / gamma
    assert err1 < 5e-4
    r2, _, tr2 = _single_electron(gamma, K, lu, substeps=2)
    u2 = tr2[:, 3:]
    gl2 = g0 * (np.sqrt(1 + np.sum(u2 * u2, axis=1)) + b0 * u2[:, 2])
    err2 = np.max(np.abs(gl2[inside] - gamma)) / gamma
    assert 3.5 < err1 / err2 < 4.5, (err1, err2)
    xs = tr[inside, 0]
    amp = 0.5 * (xs.max() - xs.min())
    beta = math.sqrt(1 - 1 / gamma ** 2)
    assert abs(amp - K / (gamma * beta * ku)) < 0.02 * K / (gamma * ku)
    # mean rest-frame drift over whole periods inside the undulator
    zi = tr[inside, 2]
    ti = t[inside]
    period_t = lu / g0 / (b0 * C0)
    nper = int((ti[-1] - ti[0]) / period_t)
    sel = ti <= ti[0] + nper * period_t
    drift = (zi[sel][-1] - zi[sel][0]) / (ti[sel][-1] - ti[sel][0]) / C0
    assert abs(drift) < 5e-3, drift


def test_optimize_bunch_position_centres_the_reference_inside_the_undulator():
    """optimize-bunch-position (Sec. MESH): the shift of the mesh is the rest-frame drift of the
    reference particle before the undulator entrance reaches it.  The electron's own trajectory
    (external field only) decides where it ends up: inside the undulator its period-averaged
    rest-frame position must be the mesh centre, up to the part of the drift that the entrance
    fringe takes away (the electron slows down over the fringe, not at the entrance).  Without
    the option it sits the whole drift ahead of the centre."""
    gamma, K, lu = 20.0, 1.0, 0.03
    res = {}
    for opt in (0, 1):
        r, w, tr = _single_electron(gamma, K, lu, steps=320, optimize=opt)
        inf = r.info()
        g0, b0, dt, dz = inf["gamma0"], inf["beta0"], inf["dt"], inf["dz"]
        n = np.arange(len(tr)) + 1
        t = inf["T0"] + (n + 0.5) * dt
        zeta = g0 * (tr[:, 2] + b0 * C0 * t)
        inside = np.nonzero(zeta > 2 * lu)[0]
        period = int(round(lu / g0 / (b0 * C0) / dt))
        assert len(inside) > 3 * period
        sel = inside[: (len(inside) // period) * period]
        centre = inf["z0"] + 0.5 * (w.nz - 1) * dz
        res[opt] = (np.mean(tr[sel, 2]) - centre) / dz, inf["z0"] / dz
    off0, z00 = res[0]
    off1, z01 = res[1]
    shift = z01 - z00                      # cells the option moved the mesh
    beta = math.sqrt(1 - 1 / gamma ** 2)
    assert shift > 5.0
    assert abs(off1) < 0.25 * shift, (off1, shift)
    assert abs(off0 - shift) < 0.25 * shift, (off0, shift)
    assert abs(off1 - (off0 - shift)) < 1e-6


def _spectrum_peak(w, steps, skip):
    """Rest-frame angular frequency of the largest peak of the on-axis E_x series (Hann window,
    zero-padded FFT, parabolic interpolation of the peak bin) after `skip` steps."""
    r = oracle.Run(oracle.params_from(w), workloads.lab_bunch(w))
    r.step(steps)
    inf = r.info()
    _, _, ex = r.series()
    seg = ex[skip:]
    seg = (seg - seg.mean()) * np.hanning(len(seg))
    nfft = 1 << 15
    spec = np.abs(np.fft.rfft(seg, nfft))
    f = np.fft.rfftfreq(nfft, inf["dt"])
    i = int(np.argmax(spec[1:])) + 1
    a, b, c = spec[i - 1], spec[i], spec[i + 1]
    di = 0.5 * (a - c) / (a - 2 * b + c)
    return 2 * math.pi * (f[i] + di * (f[1] - f[0])), inf


@pytest.mark.parametrize("kind", ["planar", "helical"])
def test_on_axis_spectrum_peaks_at_resonance(kind):
    """A cold, point-like bunch of little charge (so that its own fields do not shift its
    motion) in a 30-period static undulator radiates, in the rest frame, at w* = gamma0 beta0 c k_u;
    after the Doppler factor gamma0 (1 + beta0) the lab wavelength is the textbook resonance
    lambda_u (1 + K^2/2) / (2 gamma^2) (planar) or lambda_u (1 + K^2) / (2 gamma^2) (helical: two
    planar undulators 90 degrees and a quarter period apart, reading G9), up to O(1/gamma^2)."""
    gamma, K, lu = 20.0, 1.0, 0.03
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, und_kind=0 if kind == "planar" else 1, n_periods=30, n_particles=64,
                         sig_x=1e-6, sig_y=1e-6, sig_z=1e-6, rel_espread=0.0, space_charge=0, charge_e=1e3)
    om, inf = _spectrum_peak(w, 640, 160)
    g0, b0 = inf["gamma0"], inf["beta0"]
    ku = 2 * math.pi / lu
    assert abs(om / (g0 * b0 * C0 * ku) - 1) < 0.005
    lam_lab = 2 * math.pi * C0 / (om * g0 * (1 + b0))
    lam_res = lu * (1 + (K * K / 2 if kind == "planar" else K * K)) / (2 * gamma * gamma)
    assert abs(lam_lab / lam_res - 1) < 0.01


def test_optical_undulator_spectrum_peaks_at_inverse_compton_resonance():
    """Optical undulator (Sec. "Optical Undulator"): a counter-propagating plane wave of
    wavelength lambda_L and strength a0 (flat-top, reached after a short rise).  In the rest frame
    (gamma0 = gamma / sqrt(1 + a0^2/2)) the bunch radiates at w* = gamma0 (1 + beta0) c k_L, which
    the Doppler factor turns into the inverse-Compton wavelength lambda_L (1 + a0^2/2) / (4 gamma^2)
    in the lab.  The run is short: about 18 periods inside the wave, so the tolerance is 2 %."""
    gamma, a0, lL = 20.0, 0.5, 1e-6
    g0 = gamma / math.sqrt(1 + a0 * a0 / 2)
    b0 = math.sqrt(1 - 1 / g0 ** 2)
    dzl = lL / (g0 * (1 + b0)) / 24 / g0          # 24 cells per rest-frame radiation wavelength
    dxy = 1.5 * g0 * dzl
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, und_kind=2, K=a0, lambda_u=lL, n_periods=0, signal=1, pulse_fwhm=2 * lL,
                         dist_head=3 * lL, dx=dxy, dy=dxy, dz=dzl, gamma=gamma, n_particles=64,
                         sig_x=1e-9, sig_y=1e-9, sig_z=1e-12, rel_espread=0.0, space_charge=0, charge_e=1e3,
                         plane_dist=0.35 * 96 * dzl)
    om, inf = _spectrum_peak(w, 640, 200)
    g0, b0 = inf["gamma0"], inf["beta0"]
    assert abs(om / (g0 * (1 + b0) * C0 * 2 * math.pi / lL) - 1) < 0.02
    lam_lab = 2 * math.pi * C0 / (om * g0 * (1 + b0))
    assert abs(lam_lab / (lL * (1 + a0 * a0 / 2) / (4 * gamma * gamma)) - 1) < 0.02


@pytest.mark.parametrize("b", [0.02, 0.1])
def test_bunching_factor_inside_undulator(b):
    """A bunch modulated at the lab resonance carries that bunching in the rest frame once it
    is inside the undulator.  The instantaneous value also holds the figure-eight motion,
    a modulation travelling at 2 w*; averaging the complex bunching over one radiation
    period (two figure-eight periods) removes it, leaving the static ponderomotive bunching.
    Before the undulator the faster bunch is stretched in the rest frame (no bunching at kb)."""
    w = workloads.scaled(workloads.WORKLOADS["fel_128x128x512"], n_particles=20000, nx=8, ny=8,
                         nz=8, bunching=b, shot_noise=0, quiet=1, sig_z=3e-6, space_charge=0)
    r = oracle.Run(oracle.params_from(w), workloads.lab_bunch(w))
    _, b_before = r.diag()
    r.step(300)
    M = int(r.info()["M"])
    acc = 0j
    for _ in range(M):
        r.step(1)
        acc += r.bunching_complex()
    bf = abs(acc / M)
    # z -> z - a sin(k z) with a = 2b/k has bunching J1(2b)
    from scipy.special import j1
    assert abs(bf - j1(2 * b)) < 0.05 * b, (bf, b_before)
    assert b_before < 0.2 * b


def test_random_loading_bunching_is_noise():
    w = workloads.scaled(workloads.WORKLOADS["fel_128x128x512"], n_particles=40000, nx=8, ny=8,
                         nz=8, shot_noise=0, quiet=0)
    r = oracle.Run(oracle.params_from(w), workloads.lab_bunch(w))
    _, bf = r.diag()
    assert 0.05 / math.sqrt(40000) < bf < 5 / math.sqrt(40000)


@pytest.mark.parametrize("gamma", [1.0, 3.0])
def test_power_of_plane_wave(gamma):
    nx, ny, nz = 6, 5, 160
    lam_cells = 32
    dzl = 1.0e-4
    w = vacuum(nx, ny, nz, 3e-4, 2.5e-4, dzl, solver=0, space_charge=0, gamma=gamma)
    w = workloads.scaled(w, plane_dist=0.0)
    # the diagnostic wavelength is a rest-frame length for a run without undulator
    r0 = oracle.Run(oracle.params_from(w, periodic=(1, 1, 0)))
    dz = r0.info()["dz"]
    w = workloads.scaled(w, lambda_u=lam_cells * dz, plane_dist=(0.3 * nz * dz) / gamma)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 0)))
    inf = r.info()
    assert int(inf["M"]) == lam_cells
    k = 2 * math.pi / (lam_cells * dz)
    om = C0 * k
    a = 1.0e6
    z = inf["z0"] + np.arange(nz) * dz
    for lev, tt in ((0, 0.0), (1, inf["dt"])):
        Ax = (a / om) * np.sin(k * z - om * tt)
        r.set_field("Ax", lev, np.broadcast_to(Ax[:, None, None], (nz, ny, nx)))
    nsteps = int(inf["kp"]) - 8
    assert nsteps > lam_cells + 10
    r.step(nsteps)
    p, tl, _ = r.series()
    area = (nx - 2) * (ny - 2) * inf["dx"] * inf["dy"]
    g0, b0 = inf["gamma0"], inf["beta0"]
    # lab amplitude of a forward plane wave: E' = g0 (E_x + c b0 B_y) = g0 (1 + b0) a
    expect = (g0 * (1 + b0) * a) ** 2 / (2 * MU0 * C0) * area
    pv = p[lam_cells + 2:nsteps]
    assert np.all(np.abs(pv / expect - 1) < 0.025), (pv.min() / expect, pv.max() / expect)


def test_power_coherent_n_squared():
    base = workloads.WORKLOADS["undulator_24x24x96"]
    # low charge: trajectories are not perturbed by the self-field, so fields are linear in q
    w1 = workloads.scaled(base, n_particles=256, space_charge=0, charge_e=1e4)
    w2 = workloads.scaled(w1, charge_e=2 * w1.charge_e)
    lab = workloads.lab_bunch(w1)
    out = []
    for w in (w1, w2):
        r = oracle.Run(oracle.params_from(w), lab)
        r.step(180)
        out.append(r.series()[0])
    sel = np.abs(out[0]) > 1e-6 * np.max(np.abs(out[0]))
    assert sel.sum() > 50
    ratio = out[1][sel] / out[0][sel]
    assert np.max(np.abs(ratio - 4.0)) < 1e-3


def test_undulator_radiation_power_equals_dipole_flux():
    """One electron in a weak planar undulator (K = 0.1) oscillates harmonically in the rest frame
    at w* = gamma0 beta0 c k_u with amplitude x0, a dipole p0 = q x0.  The time-averaged Poynting
    vector of a harmonic dipole is radial with magnitude mu0 p0^2 w^4 sin^2(psi) / (32 pi^2 c r^2)
    at every distance (the near-field terms carry no mean power), psi the angle to the dipole
    axis.  Integrated over the sampling plane's interior (two rest-frame wavelengths
    downstream, 6 x 6 wavelengths), it must give the diagnostic's rest-frame power, the lab
    series over the Doppler factor gamma0^2 (1 + beta0)^2 (pinned by the plane-wave test).  x0
    comes from the velocity over one period (a constant drift from the undulator entrance drops
    out) and is checked against K / (gamma k_u).  The grid has 10 cells per rest-frame wavelength
    and a period of exactly 20 steps, so the static Coulomb field does not leak into the DFT;
    what remains is the discretisation and the Mur boundaries, 2 to 3 % here."""
    gamma, K, lu, cpl = 20.0, 0.1, 0.03, 10
    g0 = gamma / math.sqrt(1 + K * K / 2)
    b0 = math.sqrt(1 - 1 / g0 ** 2)
    lam = lu / g0
    nt = 6 * cpl
    base = workloads.WORKLOADS["undulator_24x24x96"]
    # FD Courant number such that one period is 2 cpl steps
    w = workloads.scaled(base, n_particles=1, charge_e=1.0, gamma=gamma, K=K, lambda_u=lu, n_periods=60,
                         space_charge=1, nx=nt, ny=nt, nz=8 * cpl, dx=lam / cpl, dy=lam / cpl,
                         dz=lam / (cpl * g0), solver=1, courant=math.sqrt(3) / (2 * b0), rel_espread=0.0,
                         sig_x=0.0, sig_y=0.0, sig_z=0.0, plane_dist=2 * lam / g0, dist_head=0.0)
    lab = np.array([[0.0, 0.0, 0.0, 0.0, 0.0, math.sqrt(gamma * gamma - 1)]])
    r = oracle.Run(oracle.params_from(w), lab)
    inf = r.info()
    M, dt, om = int(inf["M"]), inf["dt"], inf["omega_h"]
    assert M == 2 * cpl and abs(2 * math.pi / (om * dt) - M) < 1e-9
    steps = 10 * M
    xs, zs, vs = np.zeros(steps), np.zeros(steps), np.zeros(steps)
    for n in range(steps):
        r.step(1)
        P = r.particles()[0]
        xs[n], zs[n] = P[0], P[2]
        vs[n] = C0 * P[3] / math.sqrt(1 + P[3] ** 2 + P[4] ** 2 + P[5] ** 2)
    p, _, _ = r.series()
    prest = p / (inf["gamma0"] ** 2 * (1 + inf["beta0"]) ** 2)
    zp = inf["z0"] + inf["kp"] * inf["dz"]
    q = abs(inf["q"])
    dx, dy = inf["dx"], inf["dy"]
    sub = (np.arange(8) + 0.5) / 8 - 0.5            # 8 x 8 midpoints in every node's dx dy
    xn = (inf["x0"] + np.arange(1, nt - 1)[:, None] * dx + sub[None, :] * dx).ravel()
    yn = (inf["y0"] + np.arange(1, nt - 1)[:, None] * dy + sub[None, :] * dy).ravel()
    ratios = []
    for n in range(6 * M, steps, M // 2):
        win = np.arange(n - M + 1, n + 1)
        t = inf["T0"] + (win + 1.5) * dt
        x0 = abs((2 / M) * np.sum(vs[win] * np.exp(-1j * om * t))) / om
        assert abs(x0 / (K / (gamma * 2 * math.pi / lu)) - 1) < 0.03
        X, Y = np.meshgrid(xn - xs[win].mean(), yn, indexing="ij")
        d = zp - zs[win].mean()
        R = np.sqrt(X ** 2 + Y ** 2 + d ** 2)
        Sz = MU0 * (q * x0) ** 2 * om ** 4 / (32 * math.pi ** 2 * C0) * (1 - (X / R) ** 2) / R ** 2 * (d / R)
        ratios.append(prest[n] / (Sz.sum() * dx * dy / 64))
    ratios = np.array(ratios)
    assert len(ratios) >= 8
    assert np.all(np.abs(ratios - 1) < 0.08), ratios


def test_source_signs_coulomb_and_vector_potential():
    """An electron's potential is negative and close to Coulomb's near the charge; a slowly
    moving charge has A_z / phi = v_z / c^2 (mu0 eps0 = 1/c^2 between the two sources)."""
    nx, ny, nz = 28, 28, 40
    d = 1e-4
    w = vacuum(nx, ny, nz, d, d, d, solver=0, space_charge=1)
    w = workloads.scaled(w, charge_e=1e7)
    r0 = oracle.Run(oracle.params_from(w), np.zeros((1, 6)))
    inf = r0.info()
    D = np.array([inf["dx"], inf["dy"], inf["dz"]])
    O = np.array([inf["x0"], inf["y0"], inf["z0"]])
    beta = 0.05
    lab = np.zeros((1, 6))
    lab[0, :3] = O + np.array([13.5, 13.5, 14.5]) * D
    lab[0, 5] = beta / math.sqrt(1 - beta * beta)
    r = oracle.Run(oracle.params_from(w), lab)
    r.step(25)
    q = r.info()["q"]
    assert q < 0
    pos = r.particles()[0]
    phi = r.field("phi", 1)
    Az = r.field("Az", 1)
    X = (pos[:3] - O) / D
    i, j, k = (int(round(v)) for v in X)
    for off in (3, 4, 5, 6):
        ph = phi[k, j, i + off]
        dist = math.sqrt(((i + off - X[0]) * D[0]) ** 2 + ((j - X[1]) * D[1]) ** 2 + ((k - X[2]) * D[2]) ** 2)
        coul = q / (4 * math.pi * EPS0 * dist)
        assert ph < 0
        assert 0.7 < ph / coul < 1.3, ph / coul
        # A_z lives on the edge (k + 1/2): average the two neighbours to the node
        az = 0.5 * (Az[k, j, i + off] + Az[k - 1, j, i + off])
        assert abs(az / ph / (beta * C0 / C0 ** 2) - 1) < 0.05
