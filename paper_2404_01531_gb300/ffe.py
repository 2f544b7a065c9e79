"""ctypes binding of libffe (include/ffe.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts
Python arguments to the C structs and device pointers.  PyTorch is used for
device memory (tensors passed by data_ptr) and streams.  Loading fails loudly
when the compiled library is missing: there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libffe.so")

NV = 9
BC = {"periodic": 1, "dirichlet": 2, "no_incoming": 3, "star": 4, "outflow": 5}
ID = {"fast_wave": 0, "breakdown": 1, "cleaning_mode": 2, "wald": 3, "dipole": 4,
      "fast_wave_kink": 5, "alfven": 6, "breakdown_1d": 7}
METRIC = {"minkowski": 0, "kerr_schild": 1}
DIAG = {"l2_err": 0, "luminosity": 1, "constraints": 2, "bflux_upper": 3}
STATUS = {0: "FFE_OK", 1: "FFE_EINVAL", 2: "FFE_ENOMEM", 3: "FFE_ECUDA", 4: "FFE_ETIMEOUT",
          5: "FFE_ENUMERIC", 6: "FFE_ESTATE", 7: "FFE_ENOTIMPL"}

# every entry point declared in include/ffe.h
EXPORTS = ["ffe_create", "ffe_set_initial", "ffe_rhs", "ffe_step", "ffe_get_state", "ffe_set_state",
           "ffe_download", "ffe_upload", "ffe_get_info", "ffe_get_status", "ffe_tci_ratio",
           "ffe_near_threshold", "ffe_launch_count", "ffe_set_profiling", "ffe_profile_read",
           "ffe_fd_rhs_noalloc", "ffe_create_batch", "ffe_get_layout", "ffe_set_initial_batch",
           "ffe_rhs_vjp", "ffe_adjoint_step", "ffe_luminosity", "ffe_initial_tangent",
           "ffe_freeze_mask", "ffe_adjoint_forward", "ffe_adjoint_reverse", "ffe_save", "ffe_load",
           "ffe_constraints", "ffe_get_coords", "ffe_eval_recip", "ffe_get_mask", "ffe_set_frozen_masks",
           "ffe_diagnostic", "ffe_fp64_fma_rate",
           "ffe_last_error",
           "ffe_destroy"]


class Domain(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
                ("r_in", ctypes.c_double), ("r_out", ctypes.c_double), ("shell_ks", ctypes.c_int)]


class Elements(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3)]


class Metric(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("M", ctypes.c_double), ("a", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("kappa_psi", ctypes.c_double), ("kappa_phi", ctypes.c_double),
                ("cfl", ctypes.c_double), ("c_over_D", ctypes.c_double), ("dt", ctypes.c_double),
                ("filter_on", ctypes.c_int), ("filter_a", ctypes.c_double), ("filter_b", ctypes.c_double),
                ("tci_on", ctypes.c_int), ("tci_M", ctypes.c_int), ("tci_alpha", ctypes.c_double),
                ("weno_eps", ctypes.c_double), ("fd_corrector", ctypes.c_int),
                ("constraint_mode", ctypes.c_int), ("omega_star", ctypes.c_double), ("recon", ctypes.c_int),
                ("fd_chunk", ctypes.c_int), ("fd_capacity", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int), ("P", ctypes.c_int), ("np1", ctypes.c_int), ("nc", ctypes.c_int),
                ("n_dg", ctypes.c_int64), ("n_fd", ctypes.c_int64), ("n_state", ctypes.c_int64),
                ("dt", ctypes.c_double), ("dxmin", ctypes.c_double), ("t", ctypes.c_double),
                ("steps", ctypes.c_int64), ("n_fd_elem", ctypes.c_int), ("node_updates", ctypes.c_int64),
                ("fd_elem_updates", ctypes.c_int64), ("dg_elem_updates", ctypes.c_int64),
                ("dg_ctas_per_sm", ctypes.c_int * 3)]


_lib = None


def load():
    """Load libffe.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libffe.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "ffe_create": [ctypes.POINTER(Domain), ctypes.POINTER(Elements), i, ctypes.POINTER(Metric),
                       ctypes.POINTER(Params), P, ctypes.POINTER(P)],
        "ffe_set_initial": [P, i, ctypes.POINTER(d), i, i],
        "ffe_rhs": [P, P, P],
        "ffe_step": [P, i],
        "ffe_get_state": [P, ctypes.POINTER(P), ctypes.POINTER(P)],
        "ffe_set_state": [P, P, P],
        "ffe_download": [P, P, P],
        "ffe_upload": [P, P, P],
        "ffe_get_info": [P, ctypes.POINTER(Info)],
        "ffe_get_status": [P, ctypes.POINTER(i)],
        "ffe_tci_ratio": [P, P, P],
        "ffe_near_threshold": [P, ctypes.POINTER(i), i, ctypes.POINTER(i)],
        "ffe_launch_count": [P, ctypes.POINTER(ctypes.c_int64)],
        "ffe_set_profiling": [P, i],
        "ffe_profile_read": [P, ctypes.c_char_p, ctypes.c_size_t],
        "ffe_fd_rhs_noalloc": [i, i, ctypes.POINTER(d), d, d, i, P, P, P],
        "ffe_create_batch": [i, ctypes.POINTER(Domain), ctypes.POINTER(Elements), ctypes.POINTER(i),
                             ctypes.POINTER(Metric), ctypes.POINTER(Params), i, P, ctypes.POINTER(P)],
        "ffe_get_layout": [P, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                           ctypes.POINTER(i)],
        "ffe_set_initial_batch": [P, i, ctypes.POINTER(d), i, i],
        "ffe_rhs_vjp": [P, P, P, P, ctypes.POINTER(d)],
        "ffe_adjoint_step": [P, P, P, P, ctypes.POINTER(d)],
        "ffe_luminosity": [P, P, d, ctypes.POINTER(d), P, d],
        "ffe_initial_tangent": [P, i, P],
        "ffe_eval_recip": [P, P, ctypes.c_int64, P],
        "ffe_get_coords": [P, P, P],
        "ffe_save": [P, P, ctypes.POINTER(ctypes.c_size_t)],
        "ffe_load": [P, P, ctypes.c_size_t],
        "ffe_constraints": [P, P, ctypes.POINTER(d)],
        "ffe_get_mask": [P, ctypes.POINTER(P), ctypes.POINTER(i)],
        "ffe_set_frozen_masks": [P, i],
        "ffe_diagnostic": [P, i, ctypes.POINTER(d), ctypes.POINTER(d)],
        "ffe_fp64_fma_rate": [P, ctypes.POINTER(d)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.ffe_last_error.restype = ctypes.c_char_p
    lib.ffe_last_error.argtypes = []
    lib.ffe_destroy.argtypes = [P]
    lib.ffe_destroy.restype = None
    _lib = lib
    return lib


class FFEError(RuntimeError):
    pass


def fd_rhs_noalloc(P, Uext, h, eta, weno_eps, fd_corrector, out, stream=None):
    """FD right-hand side of caller-built extended blocks without any device
    allocation (see ffe_fd_rhs_noalloc in include/ffe.h).  Uext: contiguous
    float64 CUDA tensor [9][n][(2P+7)^3]; out: contiguous float64 CUDA tensor
    [9][n][(2P+1)^3], both on the current device (where the library resolves
    its fixed scratch array).  Sizes, types and placement are checked here,
    before the library is called, since a wrong size would make its kernels
    read or write past the buffers."""
    import torch
    ne, nc = 2 * P + 7, 2 * P + 1
    for name, t in (("Uext", Uext), ("out", out)):
        if t.dtype != torch.float64:
            raise ValueError(f"fd_rhs_noalloc: {name} must be float64, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"fd_rhs_noalloc: {name} must be contiguous")
    if Uext.numel() % (9 * ne ** 3) != 0:
        raise ValueError(f"fd_rhs_noalloc: Uext has {Uext.numel()} elements, not a multiple of 9 (2P+7)^3 = {9 * ne ** 3}")
    n = Uext.numel() // (9 * ne ** 3)
    if out.numel() != 9 * n * nc ** 3:
        raise ValueError(f"fd_rhs_noalloc: out has {out.numel()} elements, {n} blocks need 9 n (2P+1)^3 = {9 * n * nc ** 3}")
    dev = torch.cuda.current_device()
    for name, t in (("Uext", Uext), ("out", out)):
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"fd_rhs_noalloc: {name} must be a CUDA tensor on the current device cuda:{dev}")
    hh = (ctypes.c_double * 3)(*h)
    st = stream if stream is not None else torch.cuda.current_stream()
    check(load().ffe_fd_rhs_noalloc(P, n, hh, eta, weno_eps, int(fd_corrector), ctypes.c_void_p(Uext.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)))


def eval_recip(x, y, stream=None):
    """y = 1/x elementwise with the reciprocal the WENO5-Z kernels use (see
    ffe_eval_recip in include/ffe.h); x, y: float64 CUDA tensors of equal size."""
    import torch
    assert x.dtype == torch.float64 and y.dtype == torch.float64 and x.numel() == y.numel()
    st = stream if stream is not None else torch.cuda.current_stream()
    check(load().ffe_eval_recip(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(),
                                ctypes.c_void_p(st.cuda_stream)))


def fp64_fma_rate(stream=None):
    """Measured FP64 FMA throughput of the current device in TFLOP/s (see
    ffe_fp64_fma_rate in include/ffe.h)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    r = ctypes.c_double(0.0)
    check(load().ffe_fp64_fma_rate(ctypes.c_void_p(st.cuda_stream), ctypes.byref(r)))
    return r.value


def check(status):
    if status != 0:
        msg = load().ffe_last_error().decode()
        raise FFEError(f"{STATUS.get(status, status)}: {msg}")


def params_from(p):
    return Params(p["eta"], p["kappa_psi"], p["kappa_phi"], p["cfl"], p["c_over_D"], p.get("dt", 0.0),
                  p["filter_on"], p["filter_a"], p["filter_b"], p["tci_on"], p["tci_M"], p["tci_alpha"],
                  p["weno_eps"], p["fd_corrector"], p["constraint_mode"], p["omega_star"], p.get("recon", 0),
                  p.get("fd_chunk", 0), p.get("fd_capacity", 0))


class _DevArray:
    """Zero-copy CUDA-array-interface view of library-owned device memory."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3}


def domain_of(cfg):
    dom = Domain()
    el = Elements()
    if cfg["kind"] == "box":
        dom.kind = 0
        for a in range(3):
            dom.lo[a], dom.hi[a] = cfg["lo"][a], cfg["hi"][a]
            dom.bc_lo[a] = dom.bc_hi[a] = BC[cfg["bc"][a]]
            el.n[a] = cfg["n"][a]
    else:
        dom.kind = 1
        dom.r_in, dom.r_out = cfg["r_in"], cfg["r_out"]
        dom.bc_lo[0], dom.bc_hi[0] = BC[cfg["bc_inner"]], BC[cfg["bc_outer"]]
        el.n[0] = el.n[1] = cfg["n_ang"]
        el.n[2] = cfg["n_rad"]
        dom.shell_ks = 1 if cfg.get("shell_ks") else 0
    return dom, el


class Context:
    """One GRFFE problem on the current CUDA device."""

    def __init__(self, cfg, stream=None):
        import torch
        lib = load()
        self.cfg = cfg
        dom, el = domain_of(cfg)
        mk, M, spin = cfg["metric"]
        met = Metric(METRIC[mk], M, spin)
        prm = params_from(cfg["params"])
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(lib.ffe_create(ctypes.byref(dom), ctypes.byref(el), cfg["P"], ctypes.byref(met),
                             ctypes.byref(prm), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.info()

    def close(self):
        if self.h:
            load().ffe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        inf = Info()
        check(load().ffe_get_info(self.h, ctypes.byref(inf)))
        self.n_elem, self.P, self.np1, self.nc = inf.n_elem, inf.P, inf.np1, inf.nc
        self.n_dg, self.n_fd, self.n_state = inf.n_dg, inf.n_fd, inf.n_state
        self.dt, self.dxmin = inf.dt, inf.dxmin
        return inf

    def set_initial(self, kind=None, params=(), keep_mask=False, via_fd=None):
        """Analytic initial data; keep_mask: keep the current DG/FD mask (no
        indicator); via_fd: start every element on FD (default: the workload's
        "init_via_fd")."""
        if kind is None:
            kind, kw = self.cfg["initial"]
            params = tuple(kw.values())
        if via_fd is None:
            via_fd = bool(self.cfg.get("init_via_fd", False))
        arr = (ctypes.c_double * max(len(params), 1))(*params)
        flags = (1 if keep_mask else 0) | (2 if via_fd else 0)
        check(load().ffe_set_initial(self.h, ID[kind], arr, len(params), flags))

    def step(self, n=1):
        check(load().ffe_step(self.h, int(n)))

    def rhs(self, U, out):
        """U, out: float64 CUDA tensors with n_state elements."""
        check(load().ffe_rhs(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr())))

    def state(self):
        """(U, mask) as zero-copy torch views of the library's current state."""
        import torch
        pu, pm = ctypes.c_void_p(), ctypes.c_void_p()
        check(load().ffe_get_state(self.h, ctypes.byref(pu), ctypes.byref(pm)))
        U = torch.as_tensor(_DevArray(pu.value, (self.n_state,), "<f8"), device="cuda")
        m = torch.as_tensor(_DevArray(pm.value, (self.n_elem,), "|u1"), device="cuda")
        return U, m

    def set_state(self, U, mask):
        check(load().ffe_set_state(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(mask.data_ptr())))

    def download(self):
        """Host copies (numpy): U (n_state,), mask (n_elem,)."""
        U = np.empty(self.n_state)
        m = np.empty(self.n_elem, dtype=np.uint8)
        check(load().ffe_download(self.h, U.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p)))
        return U, m

    def download_into(self, U_host_ptr, mask_host_ptr=None):
        check(load().ffe_download(self.h, ctypes.c_void_p(U_host_ptr),
                                  ctypes.c_void_p(mask_host_ptr) if mask_host_ptr else None))

    def upload_from(self, U_host_ptr, mask_host_ptr=None):
        check(load().ffe_upload(self.h, ctypes.c_void_p(U_host_ptr),
                                ctypes.c_void_p(mask_host_ptr) if mask_host_ptr else None))

    def status(self):
        b = ctypes.c_int()
        check(load().ffe_get_status(self.h, ctypes.byref(b)))
        return b.value

    def tci_ratio(self, U, out):
        check(load().ffe_tci_ratio(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr())))

    def near_threshold(self):
        buf = (ctypes.c_int * 4096)()
        n = ctypes.c_int()
        check(load().ffe_near_threshold(self.h, buf, 4096, ctypes.byref(n)))
        return list(buf[:min(n.value, 4096)])

    def launch_count(self):
        n = ctypes.c_int64()
        check(load().ffe_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def set_profiling(self, on):
        check(load().ffe_set_profiling(self.h, int(bool(on))))

    def profile_read(self):
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        check(load().ffe_profile_read(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    # layout helpers: state vector <-> (9, E, ...) blocks
    def save(self):
        """Checkpoint of the context (bytes; see ffe_save in include/ffe.h)."""
        n = ctypes.c_size_t(0)
        check(load().ffe_save(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        check(load().ffe_save(self.h, buf, ctypes.byref(n)))
        return buf.raw[:n.value]

    def load_checkpoint(self, blob):
        """Restore a checkpoint made by save() on a context of the same mesh."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        check(load().ffe_load(self.h, buf, len(blob)))

    def constraints(self, U=None):
        """(max |E.B|, min (B^2 - E^2), max |psi|, max |phi|) of U (default: the state)."""
        out = (ctypes.c_double * 4)()
        check(load().ffe_constraints(self.h, ctypes.c_void_p(U.data_ptr()) if U is not None else None, out))
        return tuple(out)

    def mask(self):
        """Zero-copy torch view (uint8, n_elem) of the library's DG/FD mask."""
        import torch
        pm, n = ctypes.c_void_p(), ctypes.c_int()
        check(load().ffe_get_mask(self.h, ctypes.byref(pm), ctypes.byref(n)))
        return torch.as_tensor(_DevArray(pm.value, (n.value,), "|u1"), device="cuda")

    def set_frozen_masks(self, on=True):
        check(load().ffe_set_frozen_masks(self.h, int(bool(on))))

    def diagnostic(self, kind, args=None):
        """ffe_diagnostic: "l2_err" (args (v0, nv), default B~) -> (L2, n points),
        "luminosity" (args (r_L,)) -> (L,), "bflux_upper" (args (R,)) -> (flux,),
        "constraints" -> the 4 values of constraints().  A batched context's
        luminosity and flux take (radius, instance index)."""
        if isinstance(self, BatchContext) and kind in ("luminosity", "bflux_upper") and (not args or len(args) != 2):
            raise ValueError("a batched context's surface diagnostic takes (radius, instance)")
        if kind == "l2_err" and args is not None and len(args) != 2:
            raise ValueError("l2_err takes (v0, nv)")
        if kind in ("luminosity", "bflux_upper") and not args:
            raise ValueError(kind + " takes (radius,)")
        out = (ctypes.c_double * 4)()
        a = (ctypes.c_double * len(args))(*args) if args else None
        check(load().ffe_diagnostic(self.h, DIAG[kind], a, out))
        return {"l2_err": tuple(out[:2]), "luminosity": (out[0],), "constraints": tuple(out),
                "bflux_upper": (out[0],)}[kind]

    def coords(self):
        """(xyz_dg [3][n_dg], xyz_fd [3][n_fd]) float64 CUDA tensors: DG node and
        FD subcell-centre coordinates in state-vector order."""
        import torch
        xd = torch.empty(3 * self.n_dg, dtype=torch.float64, device="cuda")
        xf = torch.empty(3 * self.n_fd, dtype=torch.float64, device="cuda")
        check(load().ffe_get_coords(self.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(xf.data_ptr())))
        torch.cuda.synchronize()
        return xd.view(3, -1), xf.view(3, -1)

    def split(self, U):
        """(DG blocks [9][E][np1^3], FD blocks [9][E][nc^3]) of a state vector;
        with an FD slot pool the FD block of an element without a slot is zero."""
        U = np.asarray(U)
        E, np1, nc = self.n_elem, self.np1, self.nc
        dg = U[:NV * self.n_dg].reshape(NV, E, np1, np1, np1)
        if self.n_fd == E * nc ** 3:
            fd = U[NV * self.n_dg:].reshape(NV, E, nc, nc, nc)
        else:
            sl = self.layout()[1]
            pool = U[NV * self.n_dg:].reshape(NV, -1, nc, nc, nc)
            fd = np.zeros((NV, E, nc, nc, nc))
            fd[:, sl >= 0] = pool[:, sl[sl >= 0]]
        return dg, fd

    def join(self, udg, ufd):
        return np.concatenate([np.ascontiguousarray(udg).reshape(-1), np.ascontiguousarray(ufd).reshape(-1)])

    # ---- adjoint -----------------------------------------------------------
    def rhs_vjp(self, U, lam, out):
        """out = lam^T dF/dU at U; returns lam^T dF/dOmega."""
        ob = ctypes.c_double(0.0)
        check(load().ffe_rhs_vjp(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), ctypes.byref(ob)))
        return ob.value

    def adjoint_step(self, U, lam_in, lam_out):
        """lam_out = lambda_n from lambda_{n+1} for the step starting at U; returns dL/dOmega of the step."""
        ob = ctypes.c_double(0.0)
        check(load().ffe_adjoint_step(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(lam_in.data_ptr()),
                                      ctypes.c_void_p(lam_out.data_ptr()), ctypes.byref(ob)))
        return ob.value

    def adjoint_forward(self, U, stages=None, U_next=None):
        """Recompute the stages of the step from U into stages (5 state vectors:
        U2, T3, U3, T4, U4) and/or u_{n+1} into U_next."""
        vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        check(load().ffe_adjoint_forward(self.h, vp(U), vp(stages), vp(U_next)))

    def adjoint_reverse(self, U, stages, lam_in, lam_out):
        """lam_out = lambda_n from lambda_{n+1} with the stored stages of the step
        from U; returns dL/dOmega of the step."""
        ob = ctypes.c_double(0.0)
        check(load().ffe_adjoint_reverse(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(stages.data_ptr()),
                                         ctypes.c_void_p(lam_in.data_ptr()), ctypes.c_void_p(lam_out.data_ptr()),
                                         ctypes.byref(ob)))
        return ob.value

    def luminosity(self, U, r_L, grad=None, scale=1.0):
        L = ctypes.c_double(0.0)
        check(load().ffe_luminosity(self.h, ctypes.c_void_p(U.data_ptr()), float(r_L), ctypes.byref(L),
                                    ctypes.c_void_p(grad.data_ptr()) if grad is not None else None, float(scale)))
        return L.value

    def initial_tangent(self, which, out):
        check(load().ffe_initial_tangent(self.h, int(which), ctypes.c_void_p(out.data_ptr())))

    def freeze_mask(self, on=True):
        """Freeze (or release) the DG/FD mask: no indicator, no switching."""
        check(load().ffe_freeze_mask(self.h, int(bool(on))))

    def layout(self):
        """(elem_P, fd_slot, elem_inst, inst_first) as numpy arrays."""
        E = self.n_elem
        eP, sl, ei = (ctypes.c_int * E)(), (ctypes.c_int * E)(), (ctypes.c_int * E)()
        n = ctypes.c_int()
        check(load().ffe_get_layout(self.h, eP, sl, ei, None, ctypes.byref(n)))
        first = (ctypes.c_int * (n.value + 1))()
        check(load().ffe_get_layout(self.h, None, None, None, first, None))
        return np.array(eP), np.array(sl), np.array(ei), np.array(first)


class BatchContext(Context):
    """Many independent flat-space shells advanced together (ffe_create_batch)."""

    def __init__(self, cfgs, fd_capacity=0, stream=None):
        import torch
        lib = load()
        self.cfgs = cfgs
        self.cfg = cfgs[0]
        n = len(cfgs)
        doms, els = (Domain * n)(), (Elements * n)()
        prms = (Params * n)()
        Ps = (ctypes.c_int * n)(*[c["P"] for c in cfgs])
        for i, c in enumerate(cfgs):
            doms[i], els[i] = domain_of(c)
            prms[i] = params_from(c["params"])
        mk, M, spin = cfgs[0]["metric"]
        met = Metric(METRIC[mk], M, spin)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(lib.ffe_create_batch(n, doms, els, Ps, ctypes.byref(met), prms, int(fd_capacity),
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.info()

    def set_initial(self, kind=None, params=()):
        kind = self.cfgs[0]["initial"][0]
        blocks = [tuple(c["initial"][1].values()) for c in self.cfgs]
        k = len(blocks[0])
        flat = [v for b in blocks for v in b]
        arr = (ctypes.c_double * max(len(flat), 1))(*flat)
        check(load().ffe_set_initial_batch(self.h, ID[kind], arr, k, 0))

    def split_instance(self, U, i):
        """(udg, ufd, mask) of instance i from a state vector and the current layout;
        FD blocks of elements without an FD slot are zero."""
        eP, sl, ei, first = self.layout()
        E = self.n_elem
        Pm = self.P
        nns, ncs = (Pm + 1) ** 3, (2 * Pm + 1) ** 3
        dg = np.asarray(U)[:NV * self.n_dg].reshape(NV, E, nns)
        cap = self.n_fd // ncs
        fd = np.asarray(U)[NV * self.n_dg:].reshape(NV, cap, ncs)
        P = self.cfgs[i]["P"]
        np1, nc = P + 1, 2 * P + 1
        es = range(first[i], first[i + 1])
        udg = np.stack([dg[:, e, :np1 ** 3].reshape(NV, np1, np1, np1) for e in es], axis=1)
        ufd = np.stack([fd[:, sl[e], :nc ** 3].reshape(NV, nc, nc, nc) if sl[e] >= 0 else np.zeros((NV, nc, nc, nc))
                        for e in es], axis=1)
        return udg, ufd
