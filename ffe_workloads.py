"""Synthetic workload definitions shared by the tests, the benchmark and the
oracle: mesh sizes, orders, physical parameters and seeded draws.  This module
holds no arithmetic of the method; it only says which problem to set up.

Workloads (the five problem setups the library is exercised on):
  fast_wave   flat periodic cube [-1,1]^3, 4^3 elements, P=5, smooth fast wave
  breakdown   flat box [-2,2]x[-0.25,0.25]^2, 64x8x8 elements, P=5, current
              sheet that drives DG<->FD switching and the E<B clamp
  wald        Kerr-Schild M=1, a=0.9, shell r in [1.5, 50], 6 wedges x 8x8x16
  pulsars     32 rotating-dipole shells with seeded sizes and orders
  adjoint     one rotating-dipole shell, 6 wedges x 6x6x12, luminosity at r=20
  oned        the paper's 1-D tests (fast wave with kinks, stationary Alfven
              wave, FFE breakdown) at its resolutions and time steps
"""
import math

# boundary kinds and enumerations (mirrored by integer codes of the C ABI)
PERIODIC, DIRICHLET, NO_INCOMING, STAR, OUTFLOW = "periodic", "dirichlet", "no_incoming", "star", "outflow"
RELAX, HARD, RELAX_THEN_HARD = 0, 1, 2


def base_params(**kw):
    p = dict(eta=0.0, kappa_psi=1.0, kappa_phi=1.0, cfl=0.5, c_over_D=0.4186,
             filter_on=1, filter_a=36.0, filter_b=50.0, tci_on=1, tci_M=3, tci_alpha=4.0,
             weno_eps=1e-40, fd_corrector=0, constraint_mode=RELAX, omega_star=0.0)
    p.update(kw)
    return p


def fast_wave(n=4, P=5, steps=100):
    """Smooth fast wave in a periodic cube; exact solution U(x - t)."""
    return dict(name="fast_wave", kind="box", lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0),
                n=(n, n, n), bc=(PERIODIC, PERIODIC, PERIODIC), P=P,
                metric=("minkowski", 0.0, 0.0),
                params=base_params(eta=1e3, cfl=0.5),
                initial=("fast_wave", dict(amp=0.5)), steps=steps)


def breakdown(nx=64, ny=8, nz=8, P=5, steps=400, mode=RELAX, x_half=2.0):
    """FFE breakdown / current sheet: B=(1,By,0), By = 1 | -10x | -1 across
    |x|<0.1, E=(0,0,0.5) inside |x|<0.1 and (0,0,1) outside; x ends Dirichlet to
    the initial state, y and z periodic; element width 4/64 in every direction.
    Smaller variants keep the element width and shrink the box."""
    h = 2 * x_half / nx
    return dict(name="breakdown", kind="box", lo=(-x_half, -0.5 * h * ny, -0.5 * h * nz),
                hi=(x_half, 0.5 * h * ny, 0.5 * h * nz), n=(nx, ny, nz),
                bc=(DIRICHLET, PERIODIC, PERIODIC), P=P, metric=("minkowski", 0.0, 0.0),
                params=base_params(eta=1e3, cfl=0.3, fd_corrector=1, constraint_mode=mode),
                initial=("breakdown", dict()), steps=steps)


def cleaning_mode(n=4, P=5, eps=1e-3, kappa=1.0, steps=20):
    """Divergence-cleaning telegraph mode: B=(1+eps sin(pi x),0,0), E=psi=phi=q=0."""
    return dict(name="cleaning_mode", kind="box", lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0),
                n=(n, n, n), bc=(PERIODIC, PERIODIC, PERIODIC), P=P,
                metric=("minkowski", 0.0, 0.0),
                params=base_params(eta=0.0, cfl=0.5, kappa_psi=kappa, kappa_phi=kappa, tci_on=0),
                initial=("cleaning_mode", dict(eps=eps)), steps=steps)


# The paper's one-dimensional tests (Sec. IV.A, Table I, App. A): domain along
# x, time step at the lowest resolution (halved per level n) and end time.
ONED = {
    "fast_wave_kink": dict(x=(-0.5, 1.5), dt=9.22e-4, t_end=0.5),
    "alfven": dict(x=(-1.5, 1.5), dt=1.38e-3, t_end=2.0),
    "breakdown_1d": dict(x=(-0.5, 0.5), dt=4.61e-4, t_end=0.04),
}


def oned(test, n=0, P=5, via_fd=False, steps=None):
    """One of the paper's 1-D tests at resolution level n: 32 2^n elements
    along x (Dirichlet to the initial data at both ends), one element across
    [-0.1, 0.1] in y and z (periodic), eta = 1e6, CFL factor 0.3 with the
    table's time step, filter, indicator and corrector on.  via_fd: start every
    element on FD (the paper's start).  steps defaults to the test's end time."""
    o = ONED[test]
    dt = o["dt"] / 2 ** n
    return dict(name="oned_" + test, kind="box", lo=(o["x"][0], -0.1, -0.1), hi=(o["x"][1], 0.1, 0.1),
                n=(32 * 2 ** n, 1, 1), bc=(DIRICHLET, PERIODIC, PERIODIC), P=P,
                metric=("minkowski", 0.0, 0.0),
                params=base_params(eta=1e6, cfl=0.3, dt=dt, fd_corrector=1),
                initial=(test, dict()), init_via_fd=via_fd,
                steps=steps if steps is not None else int(round(o["t_end"] / dt)))


def splitmix64(seed):
    """splitmix64 stream -> uniform doubles in [0,1) (53-bit mantissa)."""
    state = seed & 0xFFFFFFFFFFFFFFFF
    while True:
        state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        z = z ^ (z >> 31)
        yield (z >> 11) * (1.0 / 9007199254740992.0)


def pulsar_draws(n_inst=32, seed=1531):
    """Per-instance draws, in order R_LC, chi, N_Omega, N_r, P."""
    g = splitmix64(seed)
    out = []
    for _ in range(n_inst):
        r_lc = 3.0 + 5.0 * next(g)
        chi = math.radians(60.0) * next(g)
        n_ang = 4 + int(5 * next(g))
        n_rad = 8 + int(9 * next(g))
        P = 4 + int(2 * next(g))
        out.append(dict(r_lc=r_lc, chi=chi, n_ang=n_ang, n_rad=n_rad, P=P))
    return out


def wald(n_ang=8, n_rad=16, P=5, r_in=1.5, r_out=50.0, spin=0.9, steps=1000):
    """Exact Wald field around a Kerr black hole (M = 1) in Kerr-Schild
    coordinates on a 6-wedge shell; Dirichlet to the exact solution at both
    radial ends; eta = 0; CFL factor 0.25."""
    return dict(name="wald", kind="shell", r_in=r_in, r_out=r_out, n_ang=n_ang, n_rad=n_rad,
                bc_inner=DIRICHLET, bc_outer=DIRICHLET, P=P, metric=("kerr_schild", 1.0, spin),
                params=base_params(eta=0.0, cfl=0.25),
                initial=("wald", dict(M=1.0, a=spin, B0=1.0)), steps=steps)


def pulsar(r_lc=6.0, chi=math.pi / 4, n_ang=6, n_rad=12, P=5, mu=1.0, r_out=None, steps=500):
    """Rotating conducting star of radius 1 with a regularised dipole (delta = 0.1)
    in flat space: star state at r = 1, no-incoming-Poynting outer boundary at
    4 R_LC (or r_out), Omega = 1/R_LC, eta = 1e5, CFL 0.25."""
    return dict(name="pulsar", kind="shell", r_in=1.0, r_out=4.0 * r_lc if r_out is None else r_out,
                n_ang=n_ang, n_rad=n_rad, bc_inner=STAR, bc_outer=NO_INCOMING, P=P,
                metric=("minkowski", 0.0, 0.0),
                params=base_params(eta=1e5, cfl=0.25, omega_star=1.0 / r_lc),
                initial=("dipole", dict(mu=mu, delta=0.1, chi=chi)), steps=steps)


def pulsars(n_inst=32, seed=1531, steps=2000):
    """The batched workload: one pulsar per seeded draw (R_LC, chi, N_Omega, N_r, P)."""
    return [pulsar(r_lc=d["r_lc"], chi=d["chi"], n_ang=d["n_ang"], n_rad=d["n_rad"], P=d["P"], steps=steps)
            for d in pulsar_draws(n_inst, seed)]


def adjoint_pulsar(tiny=False, steps=500):
    """Luminosity-gradient workload: base (mu, chi, Omega) = (1, 45 deg, 1/6),
    shell r in [1, 24] so that r = 20 is interior; 6 x 6 x 12 per wedge
    (tiny: 2 x 2 x 4)."""
    if tiny:
        return pulsar(r_lc=6.0, chi=math.pi / 4, n_ang=2, n_rad=4, r_out=24.0, steps=steps)
    return pulsar(r_lc=6.0, chi=math.pi / 4, n_ang=6, n_rad=12, r_out=24.0, steps=steps)


def wald_vacuum(spin=0.9, n_ang=4, n_rad=16, P=5, r_in=1.0, r_out=125.0, t_end=125.0):
    """The paper's vacuum Wald problem (Sec. IV.B.2): Kerr-Schild M = 1, spin a,
    Wald's magnetic field with E~ = 0 at t = 0, eta = 0, on a shell in the
    spherical Kerr-Schild radius (App. B) whose inner surface r_in = M lies
    between the two horizons, where nothing is imposed (outflow); no incoming
    Poynting flux at r_out = 125 M; 16 x 96 elements (n_rad x 6 n_ang^2) at
    P = 5, CFL factor 0.25, evolved to t_end = 125 M (a stationary state after
    t ~ 80 M).  All elements stay DG (indicator off)."""
    return dict(name="wald_vacuum", kind="shell", r_in=r_in, r_out=r_out, n_ang=n_ang, n_rad=n_rad,
                bc_inner=OUTFLOW, bc_outer=NO_INCOMING, P=P, metric=("kerr_schild", 1.0, spin),
                shell_ks=True, params=base_params(eta=0.0, cfl=0.25, tci_on=0),
                initial=("wald", dict(M=1.0, a=spin, B0=1.0, e=0.0)), t_end=t_end)
