"""Thin Python binding of libhps (include/hps.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module checks shapes,
allocates caller-owned torch tensors for the outputs and passes raw device
pointers and the current CUDA stream through ctypes.  There is no fallback:
if libhps.so is missing or no CUDA device is present, the calls raise.

Layouts (per leaf, packed leaf after leaf, row-major inside a leaf; see
include/hps.h): coefficients [6][p*p], body loads [p*p][m], S [n_i][n_b],
T [n_b][n_b], W [n_i][m], h [n_b][m], u [p*p][m], nodes [2][p*p].
"""

import ctypes
import os

import numpy as np

HPS_OK, HPS_ERR_ARG, HPS_ERR_CUDA, HPS_ERR_OOM, HPS_ERR_SINGULAR, HPS_ERR_NOCONV, HPS_ERR_STATE = range(7)
HPS_FP64, HPS_MIXED_FP32, HPS_MIXED_TF32, HPS_MIXED_BF16 = range(4)
PREC = {"fp64": HPS_FP64, "fp32": HPS_MIXED_FP32, "tf32": HPS_MIXED_TF32, "bf16": HPS_MIXED_BF16}
STATUS = {0: "HPS_OK", 1: "HPS_ERR_ARG", 2: "HPS_ERR_CUDA", 3: "HPS_ERR_OOM", 4: "HPS_ERR_SINGULAR",
          5: "HPS_ERR_NOCONV", 6: "HPS_ERR_STATE"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhps.so")


class HpsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _LeafDesc(ctypes.Structure):
    _fields_ = [("n_leaves", ctypes.c_int), ("p", ctypes.POINTER(ctypes.c_int)),
                ("box", ctypes.POINTER(ctypes.c_double)), ("kappa", ctypes.c_double)]


_lib = None


def load_library():
    """Load libhps.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhps.so not found at {LIB_PATH}; build it with "
                           "`python -m paper_2211_14969_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.hps_build_leaves.argtypes = [ctypes.POINTER(_LeafDesc), ctypes.POINTER(vp), vp]
    L.hps_leaf_nodes.argtypes = [vp, vp, vp]
    L.hps_condense.argtypes = [vp, i, vp, vp, i, d, i, vp, vp, vp, vp, vp, vp]
    L.hps_condense_host.argtypes = [vp, i, vp, vp, i, d, i, vp, vp, vp, vp, vp, i, vp]
    L.hps_merge.argtypes = [vp, i, i, vp, vp, i, vp]
    L.hps_solve.argtypes = [vp, vp, vp, vp, i, vp, vp]
    L.hps_merge_boxes.argtypes = [vp, i, i, i, i, vp, vp, i, vp, vp]
    L.hps_solve_boxes.argtypes = [vp, vp, i, vp, vp]
    L.hps_slab_factor.argtypes = [vp, i, i, i, vp, vp, i, vp]
    L.hps_slab_solve.argtypes = [vp, vp, vp, vp, i, vp, vp]
    L.hps_iti_condense.argtypes = [vp, d, vp, vp, i, vp, vp, vp, vp, vp, vp]
    L.hps_leaf_resolve.argtypes = [vp, i, vp, vp, i, vp, d, i, vp, vp, vp]
    L.hps_leaf_recover.argtypes = [vp, vp, vp, i, vp, vp, vp]
    L.hps_set_timing.argtypes = [vp, i]
    L.hps_set_blocking.argtypes = [vp, i, i]
    L.hps_set_fp64_fallback.argtypes = [vp, i]
    L.hps_set_refine_stop.argtypes = [vp, i]
    L.hps_set_merge_tensor.argtypes = [vp, i]
    L.hps_set_merge_split.argtypes = [vp, i]
    L.hps_fallback_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.hps_check_info.argtypes = [vp, vp, i, ctypes.POINTER(ctypes.c_int)]
    L.hps_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i]
    L.hps_last_launch_count.argtypes = [vp]
    L.hps_last_error.argtypes = [vp]
    L.hps_last_error.restype = ctypes.c_char_p
    L.hps_destroy.argtypes = [vp]
    L.hps_destroy.restype = None
    L.hps_version.restype = i
    for name in ("hps_build_leaves", "hps_leaf_nodes", "hps_condense", "hps_condense_host", "hps_merge", "hps_solve",
                 "hps_merge_boxes", "hps_solve_boxes", "hps_slab_factor", "hps_slab_solve", "hps_iti_condense",
                 "hps_set_timing", "hps_set_blocking", "hps_set_fp64_fallback", "hps_set_merge_split", "hps_set_refine_stop", "hps_set_merge_tensor",
                 "hps_fallback_count", "hps_check_info",
                 "hps_phase_times", "hps_last_launch_count"):
        getattr(L, name).restype = i
    _lib = L
    return L


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_dev(t, name, numel=None):
    import torch
    if t is None:
        return
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")


class Layout:
    """Packed per-leaf sizes and offsets for a list of leaf orders."""

    def __init__(self, p):
        self.p = np.asarray(p, dtype=np.int64)
        q = self.p - 2
        self.p2 = self.p * self.p
        self.ni = q * q
        self.nb = 4 * q
        self.sb = self.ni * self.nb
        self.bb = self.nb * self.nb
        self.o_p2 = np.concatenate([[0], np.cumsum(self.p2)])
        self.o_ni = np.concatenate([[0], np.cumsum(self.ni)])
        self.o_nb = np.concatenate([[0], np.cumsum(self.nb)])
        self.o_sb = np.concatenate([[0], np.cumsum(self.sb)])
        self.o_bb = np.concatenate([[0], np.cumsum(self.bb)])

    @property
    def n_leaves(self):
        return len(self.p)


class Plan:
    """An hps_plan handle (hps_build_leaves ... hps_destroy)."""

    def __init__(self, p, boxes, kappa, stream=None):
        self.handle = hps_build_leaves(p, boxes, kappa, stream)
        self.layout = Layout(p)
        self.kappa = float(kappa)

    def close(self):
        if getattr(self, "handle", None):
            load_library().hps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self):
        return load_library().hps_last_error(self.handle).decode()

    def check(self, status, what):
        if status != HPS_OK:
            raise HpsError(status, f"{what}: {self.error()}")

    def leaf_nodes(self, stream=None):
        return hps_leaf_nodes(self, stream)

    def condense(self, coef, f=None, m=None, prec="fp64", tol=1e-12, kmax=6, store_S=True,
                 store_W=True, out=None, stream=None):
        return hps_condense(self, coef, f, m, prec, tol, kmax, store_S, store_W, out, stream)

    def condense_host(self, coef, f=None, m=None, prec="fp64", tol=1e-12, kmax=6, store_S=True,
                      store_W=True, out=None, chunks=0, stream=None):
        return hps_condense_host(self, coef, f, m, prec, tol, kmax, store_S, store_W, out, chunks, stream)

    def merge(self, nx, ny, T, h, m, stream=None):
        return hps_merge(self, nx, ny, T, h, m, stream)

    def solve(self, g, S, W, m, out=None, stream=None):
        return hps_solve(self, g, S, W, m, out, stream)

    def merge_boxes(self, nx, ny, wx0, wy0, T, h, m, root=False, stream=None):
        return hps_merge_boxes(self, nx, ny, wx0, wy0, T, h, m, root, stream)

    def solve_boxes(self, g, m, out=None, stream=None):
        return hps_solve_boxes(self, g, m, out, stream)

    def slab_factor(self, nx, ny, s, T, h, m, stream=None):
        """SlabLU: slabs of s leaf columns, block LU of the interface system."""
        _check_dev(T, "T", int(self.layout.o_bb[-1]))
        self.check(load_library().hps_slab_factor(self.handle, int(nx), int(ny), int(s), _ptr(T), _ptr(h), int(m),
                                                  _stream(stream)), "hps_slab_factor")

    def iti_condense(self, coef, f=None, m=None, eta=None, store_Y=True, stream=None):
        """Impedance-to-impedance leaf maps: dict(R, h, Y, uf, info), complex
        tensors (complex128) packed like T, h, S, W."""
        import torch
        lay = self.layout
        if m is None:
            m = 0 if f is None else int(f.numel() // int(lay.o_p2[-1]))
        eta = self.kappa if eta is None else float(eta)
        _check_dev(coef, "coef", int(6 * lay.o_p2[-1]))
        _check_dev(f, "f", int(lay.o_p2[-1] * m) if f is not None else None)
        dev = coef.device
        z = lambda n: torch.empty(int(n) * 2, dtype=torch.float64, device=dev)
        o = {"R": z(lay.o_bb[-1]), "info": torch.empty(lay.n_leaves, dtype=torch.int32, device=dev)}
        if m > 0:
            o["h"] = z(lay.o_nb[-1] * m)
            o["uf"] = z(lay.o_ni[-1] * m)
        if store_Y:
            o["Y"] = z(lay.o_sb[-1])
        self.check(load_library().hps_iti_condense(self.handle, float(eta), _ptr(coef), _ptr(f), int(m), _ptr(o["R"]),
                                                   _ptr(o.get("h")), _ptr(o.get("Y")), _ptr(o.get("uf")),
                                                   _ptr(o["info"]), _stream(stream)), "hps_iti_condense")
        return {k: (torch.view_as_complex(v.view(-1, 2)) if k != "info" else v) for k, v in o.items()}

    def slab_solve(self, g, S, W, m, out=None, stream=None):
        import torch
        _check_dev(g, "g")
        _check_dev(S, "S", int(self.layout.o_sb[-1]))
        u = out if out is not None else torch.empty(int(self.layout.o_p2[-1] * m), dtype=torch.float64,
                                                    device=g.device)
        self.check(load_library().hps_slab_solve(self.handle, _ptr(g), _ptr(S), _ptr(W), int(m), _ptr(u),
                                                 _stream(stream)), "hps_slab_solve")
        return u

    def leaf_resolve(self, coef, ub, f=None, m=None, prec="fp64", tol=1e-12, kmax=6, out=None, stream=None):
        return hps_leaf_resolve(self, coef, ub, f, m, prec, tol, kmax, out, stream)

    def leaf_recover(self, S, W, ub, m, out=None, stream=None):
        return hps_leaf_recover(self, S, W, ub, m, out, stream)

    def set_blocking(self, prec, nb_panel):
        """Force the LU panel width of one precision path (0 = automatic)."""
        prec_id = PREC[prec] if isinstance(prec, str) else int(prec)
        self.check(load_library().hps_set_blocking(self.handle, prec_id, int(nb_panel)), "hps_set_blocking")

    def set_fp64_fallback(self, on=True):
        """Mixed path: re-condense non-converged leaves in FP64 (default on)."""
        self.check(load_library().hps_set_fp64_fallback(self.handle, int(bool(on))), "hps_set_fp64_fallback")

    def set_refine_stop(self, residual=True):
        """Mixed path: stop after the first correction on the true residuals
        (residual=True) or on the correction ratio alone (the default)."""
        self.check(load_library().hps_set_refine_stop(self.handle, int(bool(residual))), "hps_set_refine_stop")

    def set_merge_tensor(self, on=True):
        """The merge's large products on the tensor cores (FP64-accurate
        integer slices; True or 1, the default), also SlabLU's interface
        solves (2), or all on the FP64 pipe (False or 0)."""
        self.check(load_library().hps_set_merge_tensor(self.handle, int(on)), "hps_set_merge_tensor")

    def set_merge_split(self, below=-1):
        """Levels with fewer than `below` merges solve over many CTAs (-1: SM count; 0: never)."""
        self.check(load_library().hps_set_merge_split(self.handle, int(below)), "hps_set_merge_split")

    def check_info(self, info):
        """Host-side check of a device info tensor (hps_check_info): None when
        every entry is 0, else (status name, index of the first offending
        entry): 'HPS_ERR_SINGULAR' (exact zero pivot) before
        'HPS_ERR_NOCONV' (refinement did not converge)."""
        import torch
        if not (info.is_cuda and info.dtype == torch.int32 and info.is_contiguous()):
            raise ValueError("info must be a contiguous int32 CUDA tensor")
        first = ctypes.c_int()
        st = load_library().hps_check_info(self.handle, _ptr(info), int(info.numel()), ctypes.byref(first))
        if st == HPS_OK:
            return None
        if st in (HPS_ERR_SINGULAR, HPS_ERR_NOCONV):
            return STATUS[st], first.value
        self.check(st, "hps_check_info")

    def fallback_count(self):
        n = ctypes.c_int()
        self.check(load_library().hps_fallback_count(self.handle, ctypes.byref(n)), "hps_fallback_count")
        return n.value

    def set_timing(self, on=True):
        self.check(load_library().hps_set_timing(self.handle, int(bool(on))), "hps_set_timing")

    def phase_times(self):
        ms = (ctypes.c_float * 3)()
        self.check(load_library().hps_phase_times(self.handle, ms, 3), "hps_phase_times")
        return list(ms)

    def last_launch_count(self):
        return load_library().hps_last_launch_count(self.handle)


def hps_build_leaves(p, boxes, kappa, stream=None):
    """Build a plan; p: (n,) ints, boxes: (n, 4) x0, y0, hx, hy.  Returns the raw handle."""
    L = load_library()
    p = np.ascontiguousarray(np.asarray(p, dtype=np.int32).ravel())
    boxes = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 4))
    if boxes.shape[0] != p.shape[0]:
        raise ValueError("p and boxes disagree on the number of leaves")
    desc = _LeafDesc(int(p.shape[0]), p.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                     boxes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(kappa))
    h = ctypes.c_void_p()
    st = _stream(stream) if stream is not None or _cuda_ok() else ctypes.c_void_p(0)
    status = L.hps_build_leaves(ctypes.byref(desc), ctypes.byref(h), st)
    if status != HPS_OK:
        raise HpsError(status, L.hps_last_error(None).decode())
    return h


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def hps_leaf_nodes(plan, stream=None):
    import torch
    xy = torch.empty(int(2 * plan.layout.o_p2[-1]), dtype=torch.float64, device="cuda")
    plan.check(load_library().hps_leaf_nodes(plan.handle, _ptr(xy), _stream(stream)), "hps_leaf_nodes")
    return xy


def hps_condense(plan, coef, f=None, m=None, prec="fp64", tol=1e-12, kmax=6, store_S=True,
                 store_W=True, out=None, stream=None):
    """Condense every leaf; returns dict(S, T, h, W, info) of CUDA tensors."""
    import torch
    lay = plan.layout
    if m is None:
        m = 0 if f is None else int(f.numel() // int(lay.o_p2[-1]))
    _check_dev(coef, "coef", int(6 * lay.o_p2[-1]))
    _check_dev(f, "f", int(lay.o_p2[-1] * m) if f is not None else None)
    dev = coef.device
    o = dict(out or {})
    if "T" not in o:
        o["T"] = torch.empty(int(lay.o_bb[-1]), dtype=torch.float64, device=dev)
    if store_S and "S" not in o:
        o["S"] = torch.empty(int(lay.o_sb[-1]), dtype=torch.float64, device=dev)
    if m > 0 and "h" not in o:
        o["h"] = torch.empty(int(lay.o_nb[-1] * m), dtype=torch.float64, device=dev)
    if m > 0 and store_W and "W" not in o:
        o["W"] = torch.empty(int(lay.o_ni[-1] * m), dtype=torch.float64, device=dev)
    if "info" not in o:
        o["info"] = torch.empty(lay.n_leaves, dtype=torch.int32, device=dev)
    _check_dev(o.get("S"), "S", int(lay.o_sb[-1]))
    _check_dev(o["T"], "T", int(lay.o_bb[-1]))
    prec_id = PREC[prec] if isinstance(prec, str) else int(prec)
    status = load_library().hps_condense(
        plan.handle, prec_id, _ptr(coef), _ptr(f), int(m), float(tol), int(kmax), _ptr(o.get("S")),
        _ptr(o["T"]), _ptr(o.get("h")), _ptr(o.get("W")), _ptr(o["info"]), _stream(stream))
    plan.check(status, "hps_condense")
    return o


def _check_host(t, name, numel=None):
    if t is None:
        return
    if t.device.type != "cpu" or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous CPU tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")


def hps_condense_host(plan, coef, f=None, m=None, prec="fp64", tol=1e-12, kmax=6, store_S=True,
                      store_W=True, out=None, chunks=0, stream=None):
    """hps_condense with host (CPU) tensors in and out; copies and launches
    overlap in chunks.  Outputs are allocated pinned when not given.  The
    call is asynchronous on `stream`: synchronize before reading outputs."""
    import torch
    lay = plan.layout
    if m is None:
        m = 0 if f is None else int(f.numel() // int(lay.o_p2[-1]))
    _check_host(coef, "coef", int(6 * lay.o_p2[-1]))
    _check_host(f, "f", int(lay.o_p2[-1] * m) if f is not None else None)
    o = dict(out or {})

    def empty(n, dt=torch.float64):
        return torch.empty(int(n), dtype=dt).pin_memory()
    if "T" not in o:
        o["T"] = empty(lay.o_bb[-1])
    if store_S and "S" not in o:
        o["S"] = empty(lay.o_sb[-1])
    if m > 0 and "h" not in o:
        o["h"] = empty(lay.o_nb[-1] * m)
    if m > 0 and store_W and "W" not in o:
        o["W"] = empty(lay.o_ni[-1] * m)
    if "info" not in o:
        o["info"] = empty(lay.n_leaves, torch.int32)
    _check_host(o.get("S"), "S", int(lay.o_sb[-1]))
    _check_host(o["T"], "T", int(lay.o_bb[-1]))
    _check_host(o.get("h"), "h", int(lay.o_nb[-1] * m) if m > 0 else None)
    _check_host(o.get("W"), "W", int(lay.o_ni[-1] * m) if m > 0 else None)
    _check_host(o["info"], "info", lay.n_leaves)
    prec_id = PREC[prec] if isinstance(prec, str) else int(prec)
    status = load_library().hps_condense_host(
        plan.handle, prec_id, _ptr(coef), _ptr(f), int(m), float(tol), int(kmax), _ptr(o.get("S")),
        _ptr(o["T"]), _ptr(o.get("h")), _ptr(o.get("W")), _ptr(o["info"]), int(chunks), _stream(stream))
    plan.check(status, "hps_condense_host")
    return o


def hps_merge(plan, nx, ny, T, h, m, stream=None):
    _check_dev(T, "T", int(plan.layout.o_bb[-1]))
    status = load_library().hps_merge(plan.handle, int(nx), int(ny), _ptr(T), _ptr(h), int(m), _stream(stream))
    plan.check(status, "hps_merge")
    plan._unit_box = (1, 1)


def _box_nodes(plan, wx0, wy0):
    q = int(plan.layout.p[0]) - 2
    return 2 * (wx0 + wy0) * q


def hps_merge_boxes(plan, nx, ny, wx0, wy0, T, h, m, root=False, stream=None):
    """Merge an nx x ny grid of unit boxes of wx0 x wy0 leaves whose maps T
    ([nx*ny][nbc0][nbc0]) and fluxes h ([nx*ny][nbc0][m]) are given; with
    root=True returns the root's [T | h] (n_root x (n_root + m))."""
    import torch
    nbc0 = _box_nodes(plan, wx0, wy0)
    _check_dev(T, "T", nx * ny * nbc0 * nbc0)
    _check_dev(h, "h", nx * ny * nbc0 * m if m > 0 else None)
    th = None
    if root:
        nr = _box_nodes(plan, nx * wx0, ny * wy0)
        th = torch.empty(nr * (nr + m), dtype=torch.float64, device=T.device)
    status = load_library().hps_merge_boxes(plan.handle, int(nx), int(ny), int(wx0), int(wy0), _ptr(T), _ptr(h),
                                            int(m), _ptr(th), _stream(stream))
    plan.check(status, "hps_merge_boxes")
    plan._unit_box = (int(wx0), int(wy0))
    return th


def hps_solve_boxes(plan, g, m, out=None, stream=None):
    """Boundary values of every unit box of the last hps_merge_boxes from the
    root's Dirichlet data g: [n_boxes][nbc0][m]."""
    import torch
    _check_dev(g, "g")
    wx0, wy0 = getattr(plan, "_unit_box", (1, 1))
    n = plan.layout.n_leaves * _box_nodes(plan, wx0, wy0) * m
    ub = out if out is not None else torch.empty(n, dtype=torch.float64, device=g.device)
    _check_dev(ub, "ub", n)
    status = load_library().hps_solve_boxes(plan.handle, _ptr(g), int(m), _ptr(ub), _stream(stream))
    plan.check(status, "hps_solve_boxes")
    return ub


def hps_leaf_resolve(plan, coef, ub, f=None, m=None, prec="fp64", tol=1e-12, kmax=6, out=None, stream=None):
    """Leaf solve by re-forming and re-factoring A_ii: u at every node of
    every leaf from the edge values ub; returns dict(u, info)."""
    import torch
    lay = plan.layout
    if m is None:
        m = int(ub.numel() // int(lay.o_nb[-1]))
    _check_dev(coef, "coef", int(6 * lay.o_p2[-1]))
    _check_dev(ub, "ub", int(lay.o_nb[-1] * m))
    _check_dev(f, "f", int(lay.o_p2[-1] * m) if f is not None else None)
    o = dict(out or {})
    if "u" not in o:
        o["u"] = torch.empty(int(lay.o_p2[-1] * m), dtype=torch.float64, device=coef.device)
    if "info" not in o:
        o["info"] = torch.empty(lay.n_leaves, dtype=torch.int32, device=coef.device)
    _check_dev(o["u"], "u", int(lay.o_p2[-1] * m))
    prec_id = PREC[prec] if isinstance(prec, str) else int(prec)
    status = load_library().hps_leaf_resolve(
        plan.handle, prec_id, _ptr(coef), _ptr(f), int(m), _ptr(ub), float(tol), int(kmax), _ptr(o["u"]),
        _ptr(o["info"]), _stream(stream))
    plan.check(status, "hps_leaf_resolve")
    return o


def hps_leaf_recover(plan, S, W, ub, m, out=None, stream=None):
    """Leaf solve from stored operators: u_i = S u_b + W per leaf."""
    import torch
    lay = plan.layout
    _check_dev(S, "S", int(lay.o_sb[-1]))
    _check_dev(ub, "ub", int(lay.o_nb[-1] * m))
    u = out if out is not None else torch.empty(int(lay.o_p2[-1] * m), dtype=torch.float64, device=S.device)
    status = load_library().hps_leaf_recover(plan.handle, _ptr(S), _ptr(W), int(m), _ptr(ub), _ptr(u),
                                             _stream(stream))
    plan.check(status, "hps_leaf_recover")
    return u


def hps_solve(plan, g, S, W, m, out=None, stream=None):
    import torch
    lay = plan.layout
    _check_dev(g, "g")
    _check_dev(S, "S", int(lay.o_sb[-1]))
    u = out if out is not None else torch.empty(int(lay.o_p2[-1] * m), dtype=torch.float64, device=g.device)
    status = load_library().hps_solve(plan.handle, _ptr(g), _ptr(S), _ptr(W), int(m), _ptr(u), _stream(stream))
    plan.check(status, "hps_solve")
    return u
