"""Pins of the FP64 oracle against things other than itself.

Each test states which fact of the paper or of the mathematics it checks. The
expected values come from closed forms, from a library routine (numpy's FFT)
or from brute-force RK4 integration of the Bloch equation (Eq. 1), never from
the CUDA path.
"""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300.workloads import (GAMMA, GAMMA_BAR, Phantom, Sequence, SequenceBuilder,
                                             hard_pulse_b1, random_sequence, random_spins)

INF = np.inf


def one_spin(x=0.0, y=0.0, z=0.0, pd=1.0, t1=INF, t2=INF, dw=0.0):
    return Phantom(x=[x], y=[y], z=[z], pd=[pd], t1=[t1], t2=[t2], dw=[dw])


def hard(b, flip, tp, phase=0.0, adc=False, g=None):
    b.steps(1, tp, g_end=g, b1=hard_pulse_b1(flip, tp, phase), adc=adc)
    return b


# --------------------------------------------------------------------------
# excitation regime: Cayley-Klein rotation (spinor equations, Eq. Rot_exc)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("flip_deg", [10.0, 30.0, 90.0, 135.0, 180.0])
@pytest.mark.parametrize("phase", [0.0, np.pi / 2, -np.pi / 2, 1.1])
def test_hard_pulse_flip_angle(flip_deg, phase):
    """Hard pulse on resonance, no relaxation: Mz = M0 cos(a) and
    Mxy = i M0 sin(a) e^{i phase}. The sign follows from Eq. 1: for B1 along
    +x, dMy/dt = +gamma B1 Mz."""
    a = np.deg2rad(flip_deg)
    seq = hard(SequenceBuilder(), a, 1e-6, phase, adc=True).build()
    sig, m = oracle.simulate(one_spin(pd=0.7), seq, return_state=True)
    expect = 1j * 0.7 * np.sin(a) * np.exp(1j * phase)
    assert abs(sig[0, 0] - expect) < 1e-12
    assert abs(m[0, 2] - 0.7 * np.cos(a)) < 1e-12


def test_hard_pulses_compose_about_one_axis():
    """Two pulses about the same axis add their angles; the second one acts
    on a state with both Mxy and Mz non-zero, so every term of Eq. Rot_exc
    contributes."""
    a1, a2 = 0.7, 1.9
    b = SequenceBuilder()
    hard(b, a1, 2e-6, 0.4)
    hard(b, a2, 3e-6, 0.4, adc=True)
    sig, m = oracle.simulate(one_spin(), b.build(), return_state=True)
    assert abs(sig[0, 0] - 1j * np.sin(a1 + a2) * np.exp(0.4j)) < 1e-12
    assert abs(m[0, 2] - np.cos(a1 + a2)) < 1e-12


def test_off_resonant_rf_matches_rodrigues():
    """A constant effective field B = (B1x, B1y, Bz) rotates M about B/|B| by
    gamma|B|dt, left-handed (dM/dt = -gamma B x M). Checked against the
    Rodrigues rotation formula for that axis and angle."""
    b1 = 3e-6 * np.exp(0.3j)
    dw = 2 * np.pi * 5e3
    dt = 40e-6
    bvec = np.array([b1.real, b1.imag, dw / GAMMA])
    nrm = np.linalg.norm(bvec)
    k = bvec / nrm
    th = -GAMMA * nrm * dt

    def rot(v):
        return v * np.cos(th) + np.cross(k, v) * np.sin(th) + k * np.dot(k, v) * (1 - np.cos(th))

    # start from a tilted state: a 50 degree pulse about y, then the test step
    b = SequenceBuilder()
    hard(b, np.deg2rad(50), 1e-9, np.pi / 2)
    b.steps(1, dt, b1=b1, adc=True)
    sp = one_spin(dw=dw)
    sig, m = oracle.simulate(sp, b.build(), return_state=True)
    # state after the first (essentially instantaneous) pulse, computed with
    # the same closed form about the y axis
    s50 = np.array([-np.sin(np.deg2rad(50)), 0.0, np.cos(np.deg2rad(50))])
    # the 1 ns pulse is itself slightly off resonant; its effect is < 1e-4 rad
    v = rot(s50)
    assert abs(sig[0, 0] - (v[0] + 1j * v[1])) < 2e-4
    assert abs(m[0, 2] - v[2]) < 2e-4
    # and exactly (to 1e-10) against RK4 of Eq. 1 from the oracle's own start
    r_sig, r_m = oracle.rk4({"x": 0, "y": 0, "z": 0, "pd": 1, "t1": INF, "t2": INF, "dw": dw},
                            b.build(), substeps=4000)
    assert abs(sig[0, 0] - r_sig[0]) < 1e-10
    assert np.max(np.abs(m[0] - r_m)) < 1e-10


# --------------------------------------------------------------------------
# closed forms: FID, spin echo, Ernst steady state, k-space DFT
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dw", [0.0, 2 * np.pi * 37.0, -2 * np.pi * 120.0])
def test_fid_closed_form(dw):
    """FID after a hard pulse about -y: Mxy(t) = M0 sin(a) e^{-t/T2}
    e^{-i dw t} and Mz(t) = M0 cos(a) e^{-t/T1} + M0 (1 - e^{-t/T1}), t from
    the end of the (0.1 ns) pulse. Precession + relaxation is exact in the
    precession regime (regime-split section), so the ratio of samples is
    pinned to 1e-12 and the absolute value to the pulse's own off-resonance
    (|dw| tp <= 1e-6)."""
    a, tp, m0, T1, T2 = np.deg2rad(30), 1e-10, 0.9, 0.8, 0.05
    b = SequenceBuilder()
    hard(b, a, tp, -np.pi / 2, adc=True)
    for _ in range(50):
        b.steps(7, 1e-3 / 7)
        b.steps(1, 0.37e-3, adc=True)
    seq = b.build()
    sig, m = oracle.simulate(one_spin(pd=m0, t1=T1, t2=T2, dw=dw), seq, return_state=True)
    t = np.concatenate([[0.0], np.cumsum(seq.dt[1:])])[seq.adc[1:] == 1]
    expect = m0 * np.sin(a) * np.exp(-t / T2) * np.exp(-1j * dw * t)
    assert np.max(np.abs(sig[0] - expect)) < 2e-6
    ratio = sig[0] / sig[0, 0]
    assert np.max(np.abs(ratio - np.exp(-t / T2 - 1j * dw * t))) < 1e-12
    t_end = seq.dt[1:].sum()
    mz = m0 * np.cos(a) * np.exp(-t_end / T1) + m0 * (1 - np.exp(-t_end / T1))
    assert abs(m[0, 2] - mz) < 1e-9


@pytest.mark.parametrize("dw", [-2 * np.pi * 50, -2 * np.pi * 13.0, 0.0, 2 * np.pi * 31.0, 2 * np.pi * 50])
def test_spin_echo_refocuses(dw):
    """90x - tau - 180y - tau: the echo at TE = 2 tau is i M0 e^{-TE/T2} for
    any off-resonance, and also under a constant gradient (whose phase is
    refocused the same way). Pulses last 0.1 ns; the bound is set by the
    pulses' own off-resonance, |B_z| / |B1| < 1e-6."""
    tau, tp, T2 = 12e-3, 1e-10, 0.07
    g = np.array([0.0, 0.0, 2e-3])
    b = SequenceBuilder()
    b.steps(1, 1e-6, g)              # ramp the gradient on first
    hard(b, np.pi / 2, tp, 0.0)
    b.steps(9, tau / 9)
    hard(b, np.pi, tp, np.pi / 2)
    b.steps(13, tau / 13, adc=False)
    b.steps(1, 1e-12, adc=True)      # sample at TE
    seq = b.build()
    sp = one_spin(z=0.013, pd=1.0, t1=0.9, t2=T2, dw=dw)
    sig = oracle.simulate(sp, seq)
    te = 2 * tau + 1e-12 + 2 * tp
    assert abs(sig[0, 0] - 1j * np.exp(-te / T2)) < 1e-6


@pytest.mark.parametrize("flip_deg", [15.0, 40.0, 70.0])
def test_ernst_steady_state(flip_deg):
    """Spoiled GRE with T2 << TR reaches Mz- = M0 (1 - E1) / (1 - E1 cos a)
    and a post-pulse signal of sin(a) times that (Ernst), times the pulse's
    own transverse decay e^{-tp/T2} (rotation, then relaxation, per step)."""
    a, tr, T1, T2, m0 = np.deg2rad(flip_deg), 10e-3, 0.4, 0.5e-3, 1.3
    tp = 1e-9
    b = SequenceBuilder()
    for _ in range(300):
        hard(b, a, tp, 0.0, adc=True)
        b.steps(1, tr - tp)
    sig = oracle.simulate(one_spin(pd=m0, t1=T1, t2=T2), b.build())
    e1 = np.exp(-tr / T1)
    mz_ss = m0 * (1 - e1) / (1 - e1 * np.cos(a))
    assert abs(abs(sig[0, -1]) - np.sin(a) * mz_ss * np.exp(-tp / T2)) < 1e-8


def test_kspace_is_2d_dft():
    """No relaxation, no off-resonance, one 90x pulse, then Cartesian
    readouts: sig = i sum_j PD_j exp(-i 2 pi x_j . K) with K on the DFT grid,
    i.e. i * fftshift(fft2(ifftshift(PD))). Checks the sign of the precession
    phase, gamma, and the trapezoid integration of ramped gradients."""
    n, fov, dt = 32, 0.2, 10e-6
    rng = np.random.default_rng(7)
    img = rng.uniform(0, 1, (n, n))
    c = (np.arange(n) - n // 2) * (fov / n)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    ph = Phantom(x=xx.ravel(), y=yy.ravel(), z=np.zeros(n * n), pd=img.ravel(),
                 t1=np.full(n * n, INF), t2=np.full(n * n, INF), dw=np.zeros(n * n))
    dk, ramp = 1.0 / fov, 10
    b = SequenceBuilder()
    hard(b, np.pi / 2, 1e-6, 0.0)
    g_read = dk / (GAMMA_BAR * dt)
    for j in range(n):
        ky = (j - n // 2) * dk
        b.trapezoid([-(n // 2 + 1 + ramp / 2) * dk, ky, 0.0], ramp, 20, dt)
        b.steps(ramp, dt, [g_read, 0, 0]).steps(n, dt, adc=True).steps(ramp, dt, [0, 0, 0])
        b.trapezoid([-(n // 2 - 1 + ramp / 2) * dk, -ky, 0.0], ramp, 20, dt)
    sig = oracle.simulate(ph, b.build()).reshape(n, n)
    expect = 1j * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(img)))
    assert np.max(np.abs(sig - expect)) < 1e-9 * np.max(np.abs(expect))


# --------------------------------------------------------------------------
# brute force: RK4 on Eq. 1
# --------------------------------------------------------------------------

def _spin_dict(ph, j):
    return {k: getattr(ph, k)[j] for k in ("x", "y", "z", "pd", "t1", "t2", "dw")}


def test_precession_regime_matches_rk4():
    """With RF only in steps of constant gradient and no relaxation, the
    splitting is exact (regime-split section; hard pulses are exact, Section
    'Simulation blocks'), and so is the trapezoid phase for piecewise-linear
    gradients: oracle == RK4 to ~1e-9."""
    rng = np.random.default_rng(11)
    b = SequenceBuilder()
    hard(b, 0.9, 20e-6, 0.3)
    for _ in range(6):
        b.steps(int(rng.integers(1, 5)), float(rng.uniform(5e-6, 20e-6)),
                rng.uniform(-0.005, 0.005, 3), adc=True)
    b.steps(2, 10e-6, [0, 0, 0])
    b.steps(3, 15e-6, b1=hard_pulse_b1(0.5, 45e-6, 1.2), adc=True)  # RF at constant G = 0
    b.steps(5, 20e-6, [0.004, -0.005, 0.002], adc=True)
    seq = b.build()
    ph = random_spins(8, seed=3)
    ph.t1[:] = INF
    ph.t2[:] = INF
    for j in range(ph.n):
        sig, m = oracle.simulate(ph.subset([j]), seq, return_state=True)
        r_sig, r_m = oracle.rk4(_spin_dict(ph, j), seq, substeps=1000)
        assert np.max(np.abs(sig[0] - r_sig)) < 1e-9
        assert np.max(np.abs(m[0] - r_m)) < 1e-9


def test_relaxation_in_precession_matches_rk4():
    """In the precession regime rotation and relaxation commute, so the
    split update is exact with relaxation too (1 ps pulses keep the
    excitation's splitting error near 1e-9)."""
    rng = np.random.default_rng(12)
    b = SequenceBuilder()
    hard(b, 1.1, 1e-12, 0.3)
    for _ in range(8):
        b.steps(int(rng.integers(1, 5)), float(rng.uniform(5e-6, 20e-6)),
                rng.uniform(-0.005, 0.005, 3), adc=True)
    b.steps(1, 10e-6, [0, 0, 0])
    hard(b, 0.6, 1e-12, -0.8)
    b.steps(4, 20e-6, [0.003, 0.001, -0.004], adc=True)
    seq = b.build()
    ph = random_spins(8, seed=4)
    ph.t2[:] = rng.uniform(1e-4, 1e-3, ph.n)  # strong decay over the 0.3 ms sequence
    for j in range(ph.n):
        sig, m = oracle.simulate(ph.subset([j]), seq, return_state=True)
        r_sig, r_m = oracle.rk4(_spin_dict(ph, j), seq, substeps=1000)
        assert np.max(np.abs(sig[0] - r_sig)) < 1e-7
        assert np.max(np.abs(m[0] - r_m)) < 1e-7


def _refine(seq: Sequence, f: int) -> Sequence:
    """Same physical waveforms with every step split into f equal parts:
    B1 piecewise constant, gradient linearly interpolated; ADC kept at the
    original time points."""
    n = seq.n_steps
    dt = np.repeat(seq.dt / f, f)
    w = np.arange(1, f + 1) / f
    g = []
    for arr in (seq.gx, seq.gy, seq.gz):
        inner = (arr[:-1, None] * (1 - w[None, :]) + arr[1:, None] * w[None, :]).ravel()
        g.append(np.concatenate([[arr[0]], inner]))
    adc = np.zeros(n * f + 1, dtype=np.uint8)
    adc[0] = seq.adc[0]
    adc[f::f] = seq.adc[1:]
    return Sequence(dt, g[0], g[1], g[2], np.repeat(seq.b1, f), adc)


def test_excitation_converges_to_rk4():
    """Soft pulse with a simultaneous (time-varying) gradient and relaxation
    has no closed form. Refining the RF time step must converge to the RK4
    solution of Eq. 1; the error ratio between successive halvings gives the
    observed order (first-order splitting: global order >= 1)."""
    seq = random_sequence(40, seed=5, rf_frac=0.7, adc_frac=0.4, dt_range=(5e-6, 20e-6), g_max=0.005)
    ph = random_spins(4, seed=9)
    errs = []
    for f in (1, 2, 4, 8):
        s = _refine(seq, f)
        e = 0.0
        for j in range(ph.n):
            sig = oracle.simulate(ph.subset([j]), s)[0]
            r_sig, _ = oracle.rk4(_spin_dict(ph, j), seq, substeps=2000)
            e = max(e, np.max(np.abs(sig - r_sig)))
        errs.append(e)
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(errs[1:] < errs[:-1])
    assert np.all(order > 0.9), (errs, order)
    assert errs[-1] < 1e-3


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def test_norm_conserved_without_relaxation():
    """Rotations preserve |M| (|alpha|^2 + |beta|^2 = 1 for the spinor)."""
    seq = random_sequence(300, seed=21, rf_frac=0.5)
    ph = random_spins(50, seed=22)
    ph.t1[:] = INF
    ph.t2[:] = INF
    _, m = oracle.simulate(ph, seq, return_state=True)
    assert np.max(np.abs(np.linalg.norm(m, axis=1) - ph.pd)) < 1e-12


def test_linear_in_pd_and_additive_over_spins():
    seq = random_sequence(200, seed=31)
    ph = random_spins(64, seed=32)
    s = oracle.simulate(ph, seq)
    ph2 = random_spins(64, seed=32)
    ph2.pd *= 2.5
    s2 = oracle.simulate(ph2, seq)
    scale = np.max(np.abs(s))
    assert np.max(np.abs(s2 - 2.5 * s)) < 1e-12 * scale
    a = oracle.simulate(ph.subset(np.arange(0, 20)), seq)
    bb = oracle.simulate(ph.subset(np.arange(20, 64)), seq)
    assert np.max(np.abs(s - (a + bb))) < 1e-12 * scale


def test_split_rf_step_exact_without_relaxation():
    """A constant-field RF step equals two half steps (rotations about one
    axis compose); with relaxation it does not (splitting error)."""
    seq = random_sequence(120, seed=41, rf_frac=0.6)
    ph = random_spins(16, seed=42)
    ph.t1[:] = INF
    ph.t2[:] = INF
    # refine only steps with constant gradient: make all gradients constant
    for g in (seq.gx, seq.gy, seq.gz):
        g[:] = g[0]
    s1 = oracle.simulate(ph, seq)
    s2 = oracle.simulate(ph, _refine(seq, 2))
    assert np.max(np.abs(s1 - s2)) < 1e-11 * np.max(np.abs(s1))


def test_threads_and_groups():
    seq = random_sequence(150, seed=51)
    ph = random_spins(37, seed=52)
    s1 = oracle.simulate(ph, seq, threads=1)
    s5 = oracle.simulate(ph, seq, threads=5)
    assert np.max(np.abs(s1 - s5)) < 1e-12 * np.max(np.abs(s1))
    offs = np.array([0, 5, 5, 17, 37])
    phg = random_spins(37, seed=52)
    phg.group_offsets = offs
    sg = oracle.simulate(phg, seq, threads=3)
    assert sg.shape == (4, seq.n_adc)
    for g in range(4):
        idx = np.arange(offs[g], offs[g + 1])
        ref = oracle.simulate(ph.subset(idx), seq)[0] if len(idx) else np.zeros(seq.n_adc)
        assert np.max(np.abs(sg[g] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_degenerate_inputs():
    ph = random_spins(3, seed=61)
    empty = Sequence(np.zeros(0), np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(0, complex),
                     np.ones(1, np.uint8))
    s = oracle.simulate(ph, empty)
    assert s.shape == (1, 1) and s[0, 0] == 0  # equilibrium: no transverse magnetisation
    none = Phantom(*(np.zeros(0) for _ in range(7)))
    seq = random_sequence(10, seed=62)
    assert np.all(oracle.simulate(none, seq) == 0)


# --------------------------------------------------------------------------
# motion: x(t) = x + v t (the phantom's motion field u(x, t), Section
# "Overview"; Eq. "B definition" with G(t).x(t); the constant-velocity
# displacement of the paper's experiment (d))
# --------------------------------------------------------------------------

def moving_spin(v, **kw):
    ph = one_spin(**kw)
    ph.velocity = np.reshape(np.asarray(v, dtype=np.float64), (3, 1))
    return ph


def test_motion_zero_velocity_is_static():
    """A phantom that moves with v = 0 gives the static result."""
    seq = random_sequence(400, seed=71)
    ph = random_spins(40, seed=72)
    still = oracle.simulate(ph, seq)
    ph.velocity = np.zeros((3, ph.n))
    assert np.max(np.abs(oracle.simulate(ph, seq) - still)) < 1e-12 * np.max(np.abs(still))


@pytest.mark.parametrize("v", [0.1, -0.37, 1.5])
def test_motion_bipolar_flow_phase(v):
    """Phase-contrast flow encoding: a bipolar pair of trapezoid lobes with
    areas +A and -A, centroids T apart, has zero net area and first moment
    -A T (each lobe's moment is its area times its centroid time). A static
    spin ends with no phase; one moving at v along the gradient gets the
    phase +gamma v A T, wherever it starts."""
    g, ramp, flat = 0.02, 0.2e-3, 1.0e-3
    area = g * (flat + ramp)
    T = 2 * ramp + flat  # centroid of lobe 2 minus that of lobe 1
    b = SequenceBuilder()
    hard(b, np.pi / 2, 1e-12, 0.0)
    b.steps(1, 0.3e-3)
    for amp in (g, -g):
        b.steps(4, ramp / 4, [amp, 0, 0])
        b.steps(5, flat / 5)
        b.steps(4, ramp / 4, [0, 0, 0])
    b.steps(1, 0.1e-3, adc=True)
    seq = b.build()
    for x0 in (0.0, 0.031):
        still = oracle.simulate(one_spin(x=x0), seq)[0, 0]
        moving = oracle.simulate(moving_spin([v, 0, 0], x=x0), seq)[0, 0]
        assert abs(np.angle(still / 1j)) < 1e-8
        assert abs(moving / still - np.exp(1j * GAMMA * v * area * T)) < 1e-9
        assert abs(abs(moving) - 1.0) < 1e-12


@pytest.mark.parametrize("v", [0.1, -0.8])
def test_motion_constant_gradient_quadratic_phase(v):
    """Under a constant gradient G a spin at x0 + v t precesses at
    -gamma G (x0 + v t): its FID phase after the pulse (ending at t_p) is
    -gamma G [x0 (t - t_p) + v (t^2 - t_p^2) / 2]. Long 1 ms steps make any
    quadrature that is not exact for the quadratic integrand fail."""
    G = 0.004
    tp = 1e-12
    n = 40
    dt = np.concatenate([[tp], np.full(n, 1e-3)])
    b1 = np.zeros(n + 1, complex)
    b1[0] = hard_pulse_b1(np.pi / 2, tp)
    adc = np.concatenate([[0, 0], np.ones(n, np.uint8)])
    seq = Sequence(dt, np.full(n + 2, G), np.zeros(n + 2), np.zeros(n + 2), b1, adc)
    x0 = 0.012
    sig = oracle.simulate(moving_spin([v, 0, 0], x=x0), seq)[0]
    t = tp + 1e-3 * np.arange(1, 41)
    phase = -GAMMA * G * (x0 * (t - tp) + v * (t * t - tp * tp) / 2)
    assert np.max(np.abs(sig - 1j * np.exp(1j * phase))) < 1e-8


def test_motion_time_origin():
    """Starting the clock earlier by an idle interval T (no RF, no gradient,
    equilibrium magnetisation) with the spin T v further back is the same
    experiment."""
    seq = random_sequence(300, seed=73)
    idle = Sequence(np.full(3, 0.7e-3), np.zeros(4), np.zeros(4), np.zeros(4), np.zeros(3, complex),
                    np.zeros(4, np.uint8))
    ph = random_spins(30, seed=74)
    rng = np.random.default_rng(75)
    ph.velocity = rng.uniform(-0.5, 0.5, (3, ph.n))
    shifted = ph.subset(np.arange(ph.n))
    T = idle.duration
    shifted.x = ph.x - ph.velocity[0] * T
    shifted.y = ph.y - ph.velocity[1] * T
    shifted.z = ph.z - ph.velocity[2] * T
    seq0 = Sequence(seq.dt, seq.gx * 0 + seq.gx, seq.gy, seq.gz, seq.b1, seq.adc)
    seq0.gx[0] = seq0.gy[0] = seq0.gz[0] = 0.0  # the idle interval joins at zero gradient
    seq0 = Sequence(seq0.dt, seq0.gx, seq0.gy, seq0.gz, seq0.b1, seq0.adc)
    a = oracle.simulate(ph, seq0)
    b = oracle.simulate(shifted, idle.concat(seq0))
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(a))


def test_motion_matches_rk4():
    """Moving spins through RF (a soft pulse with a gradient) and precession
    with piecewise-linear gradients, against RK4 of Eq. 1 with x(t) = x + v t
    inside the field. Short RF steps keep the midpoint position's error below
    the bound; the precession phase is exact."""
    rng = np.random.default_rng(76)
    b = SequenceBuilder()
    b.steps(1, 1e-12, [0.0, 0.0, 0.003])
    b.steps(20, 2e-6, b1=hard_pulse_b1(0.8, 40e-6, 0.2))
    for _ in range(8):
        b.steps(int(rng.integers(1, 5)), float(rng.uniform(20e-6, 100e-6)),
                rng.uniform(-0.005, 0.005, 3), adc=True)
    b.steps(2, 40e-6, [0, 0, 0])
    b.steps(1, 1e-12, b1=hard_pulse_b1(2.0, 1e-12, 1.0))
    b.steps(6, 100e-6, [0.004, -0.005, 0.002], adc=True)
    seq = b.build()
    ph = random_spins(6, seed=77)
    # no relaxation: the soft pulse's steps are then exact rotations but for
    # the spin's motion within a step
    ph.t1[:] = INF
    ph.t2[:] = INF
    ph.velocity = rng.uniform(-1.0, 1.0, (3, ph.n))
    for j in range(ph.n):
        spin = _spin_dict(ph, j)
        spin.update(vx=ph.velocity[0, j], vy=ph.velocity[1, j], vz=ph.velocity[2, j])
        sig, m = oracle.simulate(ph.subset([j]), seq, return_state=True)
        r_sig, r_m = oracle.rk4(spin, seq, substeps=1000)
        assert np.max(np.abs(sig[0] - r_sig)) < 1e-6, j
        assert np.max(np.abs(m[0] - r_m)) < 1e-6, j
        # and the motion matters at this size
        still = oracle.simulate(Phantom(*(np.atleast_1d(spin[k]) for k in ("x", "y", "z", "pd", "t1", "t2", "dw"))),
                                seq)[0]
        assert np.max(np.abs(still - r_sig)) > 1e-2


def test_gamma_matches_the_value_the_paper_prints():
    """The oracle's gamma, read off a hard pulse's flip angle (angle = gamma
    B1 dt), agrees with the paper's printed 0.267538 rad/us/mT to its
    precision (tests/golden/gyromagnetic_ratio.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "gyromagnetic_ratio.txt")
    vals = dict(line.split() for line in open(path) if line.strip() and not line.startswith("#"))
    g_paper = float(vals["gamma_rad_per_us_per_mT"]) * 1e6 * 1e3  # rad/s/T
    tol = float(vals["relative_precision"])
    b1, tp = 1e-6, 1e-6  # T, s: a small angle, so sin(angle) ~ angle is resolved
    seq = hard(SequenceBuilder(), 0.0, tp, adc=True).build()
    seq.b1[:] = b1
    sig = oracle.simulate(one_spin(), seq)
    angle = float(np.arcsin(abs(sig[0, 0])))
    g_oracle = angle / (b1 * tp)
    assert abs(g_oracle / g_paper - 1.0) < tol
