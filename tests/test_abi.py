"""The C-ABI library builds for sm_103a and exports every entry point include/ffe.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ffe.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ffe_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2404_01531_gb300 import build, ffe
    if not os.path.exists(ffe.LIB_PATH):
        build.build()
    return ffe.LIB_PATH


def test_header_declares_the_boundary():
    names = declared()
    for n in ("ffe_create", "ffe_set_initial", "ffe_rhs", "ffe_step", "ffe_destroy", "ffe_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ffe_[a-z_0-9]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    from paper_2404_01531_gb300 import ffe
    assert sorted(ffe.EXPORTS) == declared()
    lib = ffe.load()
    for n in declared():
        assert hasattr(lib, n)


def test_library_is_device_code_for_sm_103a(lib_path):
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    assert "sm_103a" in out.stdout


def test_last_error_reports_the_last_failure(lib_path):
    """A failing call leaves its reason in ffe_last_error (thread-local),
    whatever ran before in the process."""
    import ctypes
    from paper_2404_01531_gb300 import ffe
    lib = ffe.load()
    h = ctypes.c_void_p()
    assert lib.ffe_create(None, None, 5, None, None, None, ctypes.byref(h)) == 1
    assert lib.ffe_last_error() == b"null argument"
    assert h.value is None


def _create(ffe, cfg):
    """ffe_create on a configuration, with no CUDA stream: status and message."""
    import ctypes
    lib = ffe.load()
    dom, el = ffe.domain_of(cfg)
    mk, M, spin = cfg["metric"]
    met = ffe.Metric(ffe.METRIC[mk], M, spin)
    prm = ffe.params_from(cfg["params"])
    h = ctypes.c_void_p()
    st = lib.ffe_create(ctypes.byref(dom), ctypes.byref(el), cfg["P"], ctypes.byref(met), ctypes.byref(prm),
                        None, ctypes.byref(h))
    return st, lib.ffe_last_error().decode(), h.value


PARAM_KEYS = {"eta", "kappa_psi", "kappa_phi", "cfl", "c_over_D", "dt", "filter_on", "filter_a", "filter_b",
              "tci_on", "tci_M", "tci_alpha", "weno_eps", "fd_corrector", "constraint_mode", "omega_star", "recon"}


def _bad(cfg, **kw):
    """A copy of cfg with some scheme parameters or mesh entries replaced."""
    import copy
    c = copy.deepcopy(cfg)
    for k, v in kw.items():
        (c["params"] if k in PARAM_KEYS else c)[k] = v
    return c


def test_create_rejects_invalid_configurations(lib_path):
    """ffe_create checks its whole configuration on the host before any CUDA
    call (so this runs without a GPU): each bad value is FFE_EINVAL with a
    message naming it, and no context is returned."""
    import ffe_workloads as W
    from paper_2404_01531_gb300 import ffe
    nan, inf = float("nan"), float("inf")
    box = W.breakdown(nx=4, ny=2, nz=1, x_half=0.5)
    shell = W.pulsar(r_lc=3.0, chi=0.4, n_ang=1, n_rad=4, P=5, r_out=4.0)
    cases = [
        (_bad(box, P=7), "order"),
        (_bad(box, eta=nan), "not finite"),
        (_bad(box, kappa_psi=inf), "not finite"),
        (_bad(box, eta=-1.0), "negative damping"),
        (_bad(box, dt=0.0, cfl=0.0), "need dt"),
        (_bad(box, dt=-1e-3), "need dt"),
        (_bad(box, filter_b=0.0), "filter"),
        (_bad(box, tci_alpha=0.0), "alpha"),
        (_bad(box, weno_eps=0.0), "eps"),
        (_bad(box, tci_M=9), "tci_M"),
        (_bad(box, constraint_mode=5), "constraint mode"),
        (_bad(box, recon=3), "reconstruction"),
        (_bad(box, n=[2000, 2000, 2000]), "elements"),
        (_bad(box, n=[4, 0, 1]), "elements"),
        (_bad(box, hi=[inf, 1.0, 1.0]), "not finite"),
        (_bad(box, lo=[1.0, 0.0, 0.0], hi=[1.0, 1.0, 1.0]), "empty box"),
        (_bad(shell, r_out=inf), "r_out"),
        (_bad(shell, r_in=2.0, r_out=1.0), "r_in < r_out"),
        (_bad(shell, P=6), "3 <= P <= 5"),
        (_bad(shell, n_ang=3000, n_rad=3000), "elements"),
    ]
    for cfg, what in cases:
        st, msg, h = _create(ffe, cfg)
        assert st == 1, (what, st, msg)
        assert h is None
        assert what in msg, (what, msg)


def test_create_batch_rejects_invalid_configurations(lib_path):
    """ffe_create_batch: host checks per instance before any CUDA call."""
    import ctypes
    import ffe_workloads as W
    from paper_2404_01531_gb300 import ffe
    lib = ffe.load()

    def create(cfgs, fd_capacity=0):
        n = len(cfgs)
        doms, els, prms = (ffe.Domain * max(n, 1))(), (ffe.Elements * max(n, 1))(), (ffe.Params * max(n, 1))()
        Ps = (ctypes.c_int * max(n, 1))(*[c["P"] for c in cfgs])
        for i, c in enumerate(cfgs):
            doms[i], els[i] = ffe.domain_of(c)
            prms[i] = ffe.params_from(c["params"])
        met = ffe.Metric(0, 0.0, 0.0)
        h = ctypes.c_void_p()
        st = lib.ffe_create_batch(n, doms, els, Ps, ctypes.byref(met), prms, fd_capacity, None, ctypes.byref(h))
        return st, lib.ffe_last_error().decode(), h.value

    a = W.pulsar(r_lc=3.0, chi=0.4, n_ang=1, n_rad=4, P=5, r_out=4.0)
    b = W.pulsar(r_lc=3.5, chi=0.2, n_ang=1, n_rad=6, P=4, r_out=6.0)
    for cfgs, fd_cap, what in [
        ([], 0, "bad argument"),
        ([a, b], -1, "fd_capacity"),
        ([a, _bad(b, eta=a["params"]["eta"] + 1.0)], 0, "differ"),
        ([_bad(a, eta=float("nan")), b], 0, "not finite"),
        ([a, _bad(b, P=6)], 0, "order"),
        ([a, _bad(b, r_out=float("inf"))], 0, "r_out"),
        ([a, _bad(b, n_ang=200, n_rad=200)], 0, "elements"),
    ]:
        st, msg, h = create(cfgs, fd_cap)
        assert st == 1, (what, st, msg)
        assert h is None
        assert what in msg, (what, msg)


def test_workload_configurations_pass_the_host_checks(lib_path):
    """Every workload the tests and the benchmark build gets past ffe_create's
    host checks: here (no GPU) it stops at the first device allocation, on a
    GPU the context is created and destroyed again."""
    import ctypes
    import ffe_workloads as W
    from paper_2404_01531_gb300 import ffe
    lib = ffe.load()
    wald = W.wald(n_ang=2, n_rad=2)
    wald["params"]["tci_on"] = 0
    cfgs = [W.fast_wave(), W.breakdown(nx=8, ny=2, nz=1), W.cleaning_mode(), wald, W.pulsar(n_ang=1, n_rad=2),
            W.adjoint_pulsar(tiny=True)] + [W.oned(t) for t in ("fast_wave_kink", "alfven", "breakdown_1d")]
    for cfg in cfgs:
        st, msg, h = _create(ffe, cfg)
        assert st != 1, (cfg["name"] if "name" in cfg else cfg["kind"], msg)
        if st == 0:
            lib.ffe_destroy(ctypes.c_void_p(h))
    ps = W.pulsars(n_inst=32)
    n = len(ps)
    doms, els, prms = (ffe.Domain * n)(), (ffe.Elements * n)(), (ffe.Params * n)()
    Ps = (ctypes.c_int * n)(*[c["P"] for c in ps])
    for i, c in enumerate(ps):
        doms[i], els[i] = ffe.domain_of(c)
        prms[i] = ffe.params_from(c["params"])
    h = ctypes.c_void_p()
    st = lib.ffe_create_batch(n, doms, els, Ps, ctypes.byref(ffe.Metric(0, 0.0, 0.0)), prms, 0, None, ctypes.byref(h))
    assert st != 1, lib.ffe_last_error()
    if st == 0:
        lib.ffe_destroy(h)


def test_fd_rhs_noalloc_argument_checks(lib_path):
    """ffe_fd_rhs_noalloc rejects bad orders, counts, widths, parameters and
    NULL buffers (and over-sized calls) before any CUDA call; n_elem = 0 is a
    no-op.  Runs without a GPU."""
    import ctypes
    from paper_2404_01531_gb300 import ffe
    lib = ffe.load()
    h = (ctypes.c_double * 3)(0.5, 0.5, 0.5)
    buf = ctypes.c_void_p(16)   # never dereferenced: every case below fails before a launch

    def call(P=5, n=1, hh=h, eta=0.0, eps=1e-40, U=buf, out=buf):
        return lib.ffe_fd_rhs_noalloc(P, n, hh, eta, eps, 1, U, out, None), lib.ffe_last_error().decode()

    nan = float("nan")
    cases = [dict(P=2), dict(P=7), dict(n=-1), dict(hh=None), dict(U=None), dict(out=None),
             dict(hh=(ctypes.c_double * 3)(0.5, 0.0, 0.5)), dict(hh=(ctypes.c_double * 3)(0.5, nan, 0.5)),
             dict(hh=(ctypes.c_double * 3)(float("inf"), 0.5, 0.5)), dict(eta=-1.0), dict(eta=nan),
             dict(eps=0.0), dict(eps=nan), dict(n=1000)]
    for kw in cases:
        st, msg = call(**kw)
        assert st == 1, (kw, st, msg)
        assert msg.startswith("ffe_fd_rhs_noalloc"), msg
    assert call(n=0, U=None, out=None)[0] == 0


def test_fd_rhs_noalloc_wrapper_checks_buffers_before_the_call():
    """The Python wrapper of ffe_fd_rhs_noalloc refuses, before calling the
    library, buffers whose type, layout or size would let its kernels read or
    write past them (checked here with host tensors; the size and type checks
    come before the device check)."""
    torch = pytest.importorskip("torch")
    from paper_2404_01531_gb300 import ffe
    P = 3
    ne, nc = 2 * P + 7, 2 * P + 1
    ext = torch.zeros(9 * 2 * ne ** 3, dtype=torch.float64)
    good = torch.zeros(9 * 2 * nc ** 3, dtype=torch.float64)
    with pytest.raises(ValueError, match="out has"):
        ffe.fd_rhs_noalloc(P, ext, [0.1] * 3, 0.0, 1e-40, 1, good[:-1])
    with pytest.raises(ValueError, match="not a multiple"):
        ffe.fd_rhs_noalloc(P, ext[:-1], [0.1] * 3, 0.0, 1e-40, 1, good)
    with pytest.raises(ValueError, match="float64"):
        ffe.fd_rhs_noalloc(P, ext.float(), [0.1] * 3, 0.0, 1e-40, 1, good)
    with pytest.raises(ValueError, match="contiguous"):
        ffe.fd_rhs_noalloc(P, ext, [0.1] * 3, 0.0, 1e-40, 1, torch.zeros(2 * 9 * 2 * nc ** 3, dtype=torch.float64)[::2])
    if not torch.cuda.is_available():
        with pytest.raises((ValueError, RuntimeError, AssertionError)):
            ffe.fd_rhs_noalloc(P, ext, [0.1] * 3, 0.0, 1e-40, 1, good)


def test_spherical_kerr_schild_shell_host_checks(lib_path):
    """shell_ks (the shell in the spherical Kerr-Schild radius, App. B) is a
    flag of a Kerr-Schild shell only: on a box or a flat shell it is
    FFE_EINVAL, values other than 0 and 1 are FFE_EINVAL, with the indicator
    on (FD subcells) FFE_ENOTIMPL; the vacuum Wald workload itself passes the
    host checks.  Runs without a GPU."""
    import copy
    import ctypes
    import ffe_workloads as W
    from paper_2404_01531_gb300 import ffe
    lib = ffe.load()
    ok = W.wald_vacuum(spin=0.999, n_ang=2, n_rad=2)
    st, msg, h = _create(ffe, ok)
    assert st not in (1, 7), msg
    if st == 0:
        lib.ffe_destroy(ctypes.c_void_p(h))
    flat = W.pulsar(n_ang=1, n_rad=2)
    flat["shell_ks"] = True
    assert _create(ffe, flat)[0] == 1
    box = W.fast_wave()
    box["shell_ks"] = True
    dom, el = ffe.domain_of(box)
    dom.shell_ks = 1
    met = ffe.Metric(ffe.METRIC["kerr_schild"], 1.0, 0.5)
    prm = ffe.params_from(box["params"])
    hh = ctypes.c_void_p()
    assert lib.ffe_create(ctypes.byref(dom), ctypes.byref(el), 5, ctypes.byref(met), ctypes.byref(prm), None,
                          ctypes.byref(hh)) == 1
    tci = copy.deepcopy(ok)
    tci["params"]["tci_on"] = 1
    assert _create(ffe, tci)[0] == 7
    dom2, el2 = ffe.domain_of(ok)
    dom2.shell_ks = 2
    mk, M, a = ok["metric"]
    assert lib.ffe_create(ctypes.byref(dom2), ctypes.byref(el2), 5, ctypes.byref(ffe.Metric(ffe.METRIC[mk], M, a)),
                          ctypes.byref(ffe.params_from(ok["params"])), None, ctypes.byref(hh)) == 1
