"""Python binding of libhopf_gb300 (the C ABI declared in include/hopf.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  PyTorch supplies device memory and the current stream.  There is no
CPU fallback: if the shared library is missing or fails to load, every call
raises.

Low-level names mirror the C ABI (``hopf_create``, ``hopf_eval``, ...); the
``Hopf`` class and the ``union_eval`` / ``union_closest`` / ``HopfFn`` helpers
wrap them for torch tensors.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhopf_gb300.so")

# constants of include/hopf.h
HOPF_OK, HOPF_EINVAL, HOPF_ENOMEM, HOPF_ECUDA, HOPF_ENOTSPD, HOPF_EUNSUPPORTED, HOPF_ETIMEOUT = range(7)
A_DIAG, A_DENSE = 0, 1
# initial data without a matrix: J = 1/2|x-c|_1^2 - c0, 1/2|x-c|_inf^2 - c0
J_QUAD, J_L1SQ, J_LINFSQ = 0, 2, 3
H_L1, H_WL1, H_L2, H_LINF, H_DNORM, H_ANORM = 0, 1, 2, 3, 4, 5  # H_ANORM: w = M (n x n)
P_FP64, P_FP32, P_BF16, P_SPLIT, P_MIXED = 0, 1, 2, 4, 5
STOP_PAPER, STOP_UREL = 0, 1
Q_OK, Q_NOT_CONVERGED, Q_NONFINITE, Q_ABORTED, Q_BAD_INPUT = 0, 1, 2, 3, 4

EXPORTS = ["hopf_create", "hopf_destroy", "hopf_workspace_size", "hopf_eval", "hopf_eval_f64",
           "hopf_union_workspace_size", "hopf_union_eval", "hopf_union_closest", "hopf_union_closest_noalloc",
           "hopf_backward", "hopf_backward_params", "hopf_backward_workspace_size", "hopf_backward_ws",
           "hopf_profile_events", "hopf_set_compaction", "hopf_batch_create", "hopf_batch_destroy",
           "hopf_batch_workspace_size", "hopf_batch_eval", "hopf_batch_info", "hopf_batch_set_mode",
           "hopf_eval_control", "hopf_maxH_eval",
           "hopf_measure_pipes_scratch", "hopf_measure_pipes", "hopf_set_wait_limit", "hopf_set_tc_pairs", "hopf_set_split_start",
           "hopf_set_allocator", "hopf_last_error", "hopf_version"]


class HopfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("hopf status %d: %s" % (status, msg))
        self.status = status


class hopf_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("a_kind", ctypes.c_int32), ("A", ctypes.c_void_p),
                ("centre", ctypes.c_void_p), ("c0", ctypes.c_double), ("h_kind", ctypes.c_int32),
                ("w", ctypes.c_void_p), ("lam", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32), ("stop_rule", ctypes.c_int32)]


_lib = None
_vp, _i64, _i32, _f32, _sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_size_t


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhopf_gb300.so is not built (run: python -m paper_1605_01799_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "hopf_create": ([ctypes.POINTER(hopf_desc), ctypes.POINTER(_vp), _vp], ctypes.c_int),
            "hopf_destroy": ([_vp], None),
            "hopf_workspace_size": ([_vp, _i64, ctypes.POINTER(_sz)], ctypes.c_int),
            "hopf_eval": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
            "hopf_eval_f64": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
            "hopf_union_workspace_size": ([_vp, _i32, _i64, ctypes.POINTER(_sz)], ctypes.c_int),
            "hopf_union_eval": ([_vp, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
            "hopf_union_closest": ([_vp, _i32, _i64, _vp, _f32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp],
                                   ctypes.c_int),
            "hopf_union_closest_noalloc": ([_vp, _i32, _i64, _vp, _f32, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
                                           ctypes.c_int),
            "hopf_backward": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
            "hopf_backward_params": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
            "hopf_backward_workspace_size": ([_vp, _i64, ctypes.POINTER(_sz)], ctypes.c_int),
            "hopf_backward_ws": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
            "hopf_profile_events": ([_vp, _vp, _vp], ctypes.c_int),
            "hopf_set_compaction": ([_vp, _i32], ctypes.c_int),
            "hopf_batch_create": ([ctypes.POINTER(hopf_desc), _i32, ctypes.POINTER(_vp), _vp], ctypes.c_int),
            "hopf_batch_destroy": ([_vp], None),
            "hopf_batch_workspace_size": ([_vp, _vp, ctypes.POINTER(_sz)], ctypes.c_int),
            "hopf_batch_eval": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
            "hopf_batch_info": ([_vp, _vp, _vp, _vp], ctypes.c_int),
            "hopf_batch_set_mode": ([_vp, _i32], ctypes.c_int),
            "hopf_eval_control": ([_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp],
                                  ctypes.c_int),
            "hopf_maxH_eval": ([_vp, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
            "hopf_set_wait_limit": ([_vp, _i64], ctypes.c_int),
            "hopf_set_tc_pairs": ([_vp, ctypes.c_int32], ctypes.c_int),
            "hopf_set_split_start": ([_vp, ctypes.c_double], ctypes.c_int),
            "hopf_set_allocator": ([_vp, _vp, _vp], ctypes.c_int),
            "hopf_measure_pipes_scratch": ([], _sz),
            "hopf_measure_pipes": ([_vp, _sz, _vp, _vp, _vp, _vp], ctypes.c_int),
            "hopf_last_error": ([], ctypes.c_char_p),
            "hopf_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != HOPF_OK:
        raise HopfError(status, lib().hopf_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def version():
    return lib().hopf_version().decode()


def measure_pipes(stream=None):
    """Measured FP32 and FP64 FMA throughput (TFLOP/s) and L2 read bandwidth
    (GB/s) of the current device, from the library's probe kernels."""
    import torch
    buf = torch.empty(int(lib().hopf_measure_pipes_scratch()), dtype=torch.uint8, device="cuda")
    f32, f64, l2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().hopf_measure_pipes(_ptr(buf), buf.numel(), ctypes.byref(f32), ctypes.byref(f64), ctypes.byref(l2),
                                    _stream(stream)))
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value, "l2_read_gbs": l2.value}


def _a_kind(A, j_kind, n):
    """(A as float64 or None, desc a_kind, n) for a quadratic J (A given) or a
    norm J (j_kind, n given)."""
    if int(j_kind) != J_QUAD:
        assert A is None and n is not None, "a norm J takes n and no A"
        return None, int(j_kind), int(n)
    A = np.ascontiguousarray(A, dtype=np.float64)
    return A, (A_DIAG if A.ndim == 1 else A_DENSE), A.shape[0]


class Hopf:
    """One problem instance: J(x) = 1/2 (x-c)^T A^{-1} (x-c) - c0 with A
    diagonal (1-D ``A``) or dense (2-D ``A``), or with ``A=None``,
    ``j_kind`` J_L1SQ / J_LINFSQ and ``n``, J = 1/2|x-c|_1^2 - c0 or
    1/2|x-c|_inf^2 - c0; H one of H_L1, H_WL1, H_L2, H_LINF, H_DNORM and
    H_ANORM (sqrt(<p, M p>), ``w`` = M, n x n)."""

    def __init__(self, A, h_kind, w=None, centre=None, c0=0.5, lam=1.0, tol=1e-14, max_iter=1000,
                 precision=P_FP32, stop_rule=STOP_UREL, stream=None, j_kind=J_QUAD, n=None):
        import torch  # noqa: F401  (device context)
        A, self.a_kind, self.n = _a_kind(A, j_kind, n)
        self.j_kind = int(j_kind)
        self.h_kind, self.precision = int(h_kind), int(precision)
        self._keep = [A]
        wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        cv = None if centre is None else np.ascontiguousarray(centre, dtype=np.float64)
        self._keep += [wv, cv]
        d = hopf_desc(self.n, self.a_kind, None if A is None else A.ctypes.data,
                      None if cv is None else cv.ctypes.data, float(c0),
                      self.h_kind, None if wv is None else wv.ctypes.data, float(lam), float(tol), int(max_iter),
                      self.precision, int(stop_rule))
        h = ctypes.c_void_p()
        _check(lib().hopf_create(ctypes.byref(d), ctypes.byref(h), _stream(stream)))
        self.handle = h
        self._ws = None

    def close(self):
        if getattr(self, "handle", None):
            lib().hopf_destroy(self.handle)
            self.handle = None

    __del__ = close

    def workspace_size(self, batch):
        b = ctypes.c_size_t()
        _check(lib().hopf_workspace_size(self.handle, int(batch), ctypes.byref(b)))
        return b.value

    def workspace(self, batch):
        import torch
        need = self.workspace_size(batch)
        if need == 0:
            return None
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        return self._ws

    def eval(self, x, t, out=None, workspace=None, stream=None):
        """x: [B, n] float32 cuda, t: [B] float32 cuda.  Returns a dict of
        phi (float64), grad, dphidt, iters (int32), status (uint8)."""
        import torch
        fp64 = self.precision == P_FP64
        dt = torch.float64 if fp64 else torch.float32
        assert x.dtype == dt and t.dtype == dt and x.is_cuda and x.is_contiguous() and t.is_contiguous()
        B = x.shape[0]
        if out is None:
            out = {"phi": torch.empty(B, dtype=torch.float64, device=x.device),
                   "grad": torch.empty(B, self.n, dtype=dt, device=x.device),
                   "dphidt": torch.empty(B, dtype=dt, device=x.device),
                   "iters": torch.empty(B, dtype=torch.int32, device=x.device),
                   "status": torch.empty(B, dtype=torch.uint8, device=x.device)}
        ws = workspace if workspace is not None else self.workspace(B)
        nbytes = 0 if ws is None else ws.numel()
        f = lib().hopf_eval_f64 if fp64 else lib().hopf_eval
        _check(f(self.handle, B, _ptr(x), _ptr(t), _ptr(out["phi"]), _ptr(out["grad"]), _ptr(out.get("dphidt")),
                 _ptr(out.get("iters")), _ptr(out.get("status")), _ptr(ws), nbytes, _stream(stream)))
        return out

    def eval_control(self, x, t, out=None, workspace=None, stream=None):
        """eval plus the optimal control beta in dH(grad phi) and the terminal
        point x_final = x - t beta (Section 2), both [B, n] float32."""
        import torch
        assert x.dtype == torch.float32 and t.dtype == torch.float32 and x.is_cuda
        B = x.shape[0]
        if out is None:
            out = {"phi": torch.empty(B, dtype=torch.float64, device=x.device),
                   "grad": torch.empty(B, self.n, dtype=torch.float32, device=x.device),
                   "dphidt": torch.empty(B, dtype=torch.float32, device=x.device),
                   "iters": torch.empty(B, dtype=torch.int32, device=x.device),
                   "status": torch.empty(B, dtype=torch.uint8, device=x.device),
                   "beta": torch.empty(B, self.n, dtype=torch.float32, device=x.device),
                   "x_final": torch.empty(B, self.n, dtype=torch.float32, device=x.device)}
        ws = workspace if workspace is not None else self.workspace(B)
        nbytes = 0 if ws is None else ws.numel()
        _check(lib().hopf_eval_control(self.handle, B, _ptr(x), _ptr(t), _ptr(out["phi"]), _ptr(out["grad"]),
                                       _ptr(out.get("dphidt")), _ptr(out.get("iters")), _ptr(out.get("status")),
                                       _ptr(out["beta"]), _ptr(out.get("x_final")), _ptr(ws), nbytes,
                                       _stream(stream)))
        return out

    def profile_events(self, start=None, stop=None):
        """Record torch.cuda.Event pair around the main solver kernel of later
        eval calls (None, None turns it off)."""
        sp = None if start is None else ctypes.c_void_p(start.cuda_event)
        ep = None if stop is None else ctypes.c_void_p(stop.cuda_event)
        _check(lib().hopf_profile_events(self.handle, sp, ep))

    def set_wait_limit(self, cycles):
        """Clock-cycle limit of the dense solvers' bounded waits (0: default)."""
        _check(lib().hopf_set_wait_limit(self.handle, int(cycles)))

    def set_split_start(self, tol_switch):
        """MIXED form (l1, weighted l1): SPLIT iterations until each query's
        squared relative change is within tol_switch, then the defect
        correction to the tolerance; 0 runs the defect correction alone."""
        _check(lib().hopf_set_split_start(self.handle, float(tol_switch)))

    def set_tc_pairs(self, on):
        """Dense tensor-core path: SM pairs (cta_group::2) on or off."""
        _check(lib().hopf_set_tc_pairs(self.handle, 1 if on else 0))

    def set_compaction(self, on):
        _check(lib().hopf_set_compaction(self.handle, 1 if on else 0))

    def backward(self, g_phi, vstar, want_x=True, want_t=True, want_A=True, stream=None, tensor_cores=True):
        """Envelope-theorem gradients (hopf_backward).  For a dense A, g_A runs
        on the tensor cores (hopf_backward_ws, with a workspace kept between
        calls of the same batch size) unless tensor_cores is False, which
        selects the FP32 CUDA-core kernel."""
        import torch
        B = vstar.shape[0]
        gx = torch.empty_like(vstar) if want_x else None
        gt = torch.empty(B, dtype=torch.float32, device=vstar.device) if want_t else None
        gA = None
        if want_A and self.j_kind == J_QUAD:  # a norm J has no matrix
            shape = (self.n, self.n) if self.a_kind == A_DENSE else (self.n,)
            gA = torch.empty(shape, dtype=torch.float32, device=vstar.device)
        if gA is not None and self.a_kind == A_DENSE and B > 0 and tensor_cores:
            b = ctypes.c_size_t()
            _check(lib().hopf_backward_workspace_size(self.handle, B, ctypes.byref(b)))
            ws = getattr(self, "_bwd_ws", None)
            if ws is None or ws.numel() < b.value or ws.device != vstar.device:
                ws = self._bwd_ws = torch.empty(b.value, dtype=torch.uint8, device=vstar.device)
            _check(lib().hopf_backward_ws(self.handle, B, _ptr(g_phi), _ptr(vstar), _ptr(gx), _ptr(gt), _ptr(gA),
                                          _ptr(ws), ws.numel(), _stream(stream)))
            return gx, gt, gA
        _check(lib().hopf_backward(self.handle, B, _ptr(g_phi), _ptr(vstar), _ptr(gx), _ptr(gt), _ptr(gA),
                                   _stream(stream)))
        return gx, gt, gA

    def backward_params(self, g_phi, vstar, t=None, dphidt=None, want_c=True, want_c0=True, want_w=False,
                        stream=None):
        """dL/dc [n], dL/dc0 [1] and dL/dw [n] of L = sum_q g_phi[q] phi_q
        (envelope theorem; dL/dw for the weighted Hamiltonians, which needs t,
        and dphidt for sqrt(sum w p^2))."""
        import torch
        B = vstar.shape[0]
        dev = vstar.device
        gc = torch.empty(self.n, dtype=torch.float32, device=dev) if want_c else None
        gc0 = torch.empty(1, dtype=torch.float32, device=dev) if want_c0 else None
        gw = torch.empty(self.n, dtype=torch.float32, device=dev) if want_w else None
        _check(lib().hopf_backward_params(self.handle, B, _ptr(g_phi), _ptr(vstar), _ptr(t), _ptr(dphidt),
                                          _ptr(gc), _ptr(gc0), _ptr(gw), _stream(stream)))
        return gc, gc0, gw


class HopfBatch:
    """A ragged batch of instances evaluated as one CUDA graph replay.
    ``instances``: list of dicts with keys A (1-D diagonal or 2-D dense; or
    None with j_kind and n), h_kind and optionally w, centre, c0, lam, tol,
    max_iter, precision, stop_rule (as for Hopf)."""

    def __init__(self, instances, stream=None):
        self._keep = []
        descs = (hopf_desc * len(instances))()
        self.ns = []
        for i, d in enumerate(instances):
            A, a_kind, n = _a_kind(d.get("A"), d.get("j_kind", J_QUAD), d.get("n"))
            w = d.get("w")
            w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
            c = d.get("centre")
            c = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
            self._keep += [A, w, c]
            descs[i] = hopf_desc(n, a_kind, None if A is None else A.ctypes.data,
                                 None if c is None else c.ctypes.data, float(d.get("c0", 0.5)), int(d["h_kind"]),
                                 None if w is None else w.ctypes.data, float(d.get("lam", 1.0)),
                                 float(d.get("tol", 1e-13)), int(d.get("max_iter", 1000)),
                                 int(d.get("precision", P_MIXED if a_kind == A_DENSE else P_FP32)),
                                 int(d.get("stop_rule", STOP_UREL)))
            self.ns.append(n)
        h = ctypes.c_void_p()
        _check(lib().hopf_batch_create(descs, len(instances), ctypes.byref(h), _stream(stream)))
        self.handle = h
        self._ws = None

    def close(self):
        if getattr(self, "handle", None):
            lib().hopf_batch_destroy(self.handle)
            self.handle = None

    __del__ = close

    def eval(self, counts, x, t, out=None, stream=None):
        """counts: per-instance query counts; x: flat float32 cuda tensor of
        sum(counts[i] * n_i) values; t: float32 [sum(counts)]."""
        import torch
        cnt = np.ascontiguousarray(counts, dtype=np.int64)
        Q = int(cnt.sum())
        X = int((cnt * np.array(self.ns, dtype=np.int64)).sum())
        assert x.numel() == X and t.numel() == Q
        if out is None:
            out = {"phi": torch.empty(Q, dtype=torch.float64, device=x.device),
                   "grad": torch.empty(X, dtype=torch.float32, device=x.device),
                   "dphidt": torch.empty(Q, dtype=torch.float32, device=x.device),
                   "iters": torch.empty(Q, dtype=torch.int32, device=x.device),
                   "status": torch.empty(Q, dtype=torch.uint8, device=x.device)}
        b = ctypes.c_size_t()
        _check(lib().hopf_batch_workspace_size(self.handle, cnt.ctypes.data, ctypes.byref(b)))
        if self._ws is None or self._ws.numel() < max(b.value, 1):
            self._ws = torch.empty(max(b.value, 1), dtype=torch.uint8, device=x.device)
        _check(lib().hopf_batch_eval(self.handle, cnt.ctypes.data, _ptr(x), _ptr(t), _ptr(out["phi"]),
                                     _ptr(out["grad"]), _ptr(out["dphidt"]), _ptr(out["iters"]),
                                     _ptr(out["status"]), _ptr(self._ws), self._ws.numel(), _stream(stream)))
        return out

    def info(self):
        ns, ug = ctypes.c_int32(), ctypes.c_int32()
        ms = (ctypes.c_float * 8)()
        _check(lib().hopf_batch_info(self.handle, ctypes.byref(ns), ctypes.byref(ug), ms))
        return {"nstreams": ns.value, "used_graph": bool(ug.value), "tuned_ms": list(ms),
                "schedule": {0: None, 1: "persistent", 2: "streams"}[ug.value]}

    def set_mode(self, mode):
        """0: the tuner picks the persistent or the stream schedule; 1: the
        persistent one only; 2: the streams only."""
        _check(lib().hopf_batch_set_mode(self.handle, int(mode)))


def _parts_array(parts):
    arr = (ctypes.c_void_p * len(parts))(*[p.handle.value for p in parts])
    return arr


def _union_ws(arr, K, B, device, workspace):
    import torch
    b = ctypes.c_size_t()
    _check(lib().hopf_union_workspace_size(arr, K, B, ctypes.byref(b)))
    if workspace is not None and workspace.numel() >= b.value:
        return workspace
    return torch.empty(max(b.value, 1), dtype=torch.uint8, device=device)


def union_eval(parts, x, t, out=None, workspace=None, stream=None):
    """phi = min_i phi_i over diagonal parts (Section 2.2).  ``out`` (a dict
    returned by an earlier call) and ``workspace`` may be passed back in to
    reuse their buffers."""
    import torch
    B, n = x.shape
    arr = _parts_array(parts)
    ws = _union_ws(arr, len(parts), B, x.device, workspace)
    if out is None:
        out = {"phi": torch.empty(B, dtype=torch.float64, device=x.device),
               "grad": torch.empty(B, n, dtype=torch.float32, device=x.device),
               "argmin": torch.empty(B, dtype=torch.int32, device=x.device),
               "iters": torch.empty(B, dtype=torch.int32, device=x.device),
               "status": torch.empty(B, dtype=torch.uint8, device=x.device)}
    out["workspace"] = ws
    _check(lib().hopf_union_eval(arr, len(parts), B, _ptr(x), _ptr(t), _ptr(out["phi"]), _ptr(out["grad"]),
                                 _ptr(out["argmin"]), _ptr(out["iters"]), _ptr(out["status"]), _ptr(ws), ws.numel(),
                                 _stream(stream)))
    return out


def maxH_eval(parts, x, t, out=None, workspace=None, stream=None):
    """phi = max_i phi_i over diagonal parts that share J and differ in H
    (Section 2.2: the solution for the Hamiltonian min_i H_i)."""
    import torch
    B, n = x.shape
    arr = _parts_array(parts)
    ws = _union_ws(arr, len(parts), B, x.device, workspace)
    if out is None:
        out = {"phi": torch.empty(B, dtype=torch.float64, device=x.device),
               "grad": torch.empty(B, n, dtype=torch.float32, device=x.device),
               "argmax": torch.empty(B, dtype=torch.int32, device=x.device),
               "iters": torch.empty(B, dtype=torch.int32, device=x.device),
               "status": torch.empty(B, dtype=torch.uint8, device=x.device)}
    out["workspace"] = ws
    _check(lib().hopf_maxH_eval(arr, len(parts), B, _ptr(x), _ptr(t), _ptr(out["phi"]), _ptr(out["grad"]),
                                _ptr(out["argmax"]), _ptr(out["iters"]), _ptr(out["status"]), _ptr(ws), ws.numel(),
                                _stream(stream)))
    return out


def union_closest(parts, x, s_tol=1e-6, max_newton=50, out=None, workspace=None, stream=None):
    """Distance and closest point to the union of {J_i <= 0} (Section 3.2).
    ``out`` and ``workspace`` as for union_eval."""
    import torch
    B, n = x.shape
    arr = _parts_array(parts)
    ws = _union_ws(arr, len(parts), B, x.device, workspace)
    if out is None:
        out = {"dist": torch.empty(B, dtype=torch.float32, device=x.device),
               "closest": torch.empty(B, n, dtype=torch.float32, device=x.device),
               "argmin": torch.empty(B, dtype=torch.int32, device=x.device),
               "newton": torch.empty(B, dtype=torch.int32, device=x.device),
               "status": torch.empty(B, dtype=torch.uint8, device=x.device)}
    out["workspace"] = ws
    _check(lib().hopf_union_closest(arr, len(parts), B, _ptr(x), float(s_tol), int(max_newton), _ptr(out["dist"]),
                                    _ptr(out["closest"]), _ptr(out["argmin"]), _ptr(out["newton"]),
                                    _ptr(out["status"]), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def union_closest_noalloc(parts, x, s_tol=1e-6, max_newton=50, out=None, stream=None):
    """union_closest without allocation inside the library (static scratch of
    8 MiB: batch * len(parts) up to about 490,000).  Pass preallocated
    ``out`` tensors to keep the whole call allocation-free."""
    import torch
    B, n = x.shape
    arr = _parts_array(parts)
    if out is None:
        out = {"dist": torch.empty(B, dtype=torch.float32, device=x.device),
               "closest": torch.empty(B, n, dtype=torch.float32, device=x.device),
               "argmin": torch.empty(B, dtype=torch.int32, device=x.device),
               "newton": torch.empty(B, dtype=torch.int32, device=x.device),
               "status": torch.empty(B, dtype=torch.uint8, device=x.device)}
    _check(lib().hopf_union_closest_noalloc(arr, len(parts), B, _ptr(x), float(s_tol), int(max_newton),
                                            _ptr(out["dist"]), _ptr(out["closest"]), _ptr(out["argmin"]),
                                            _ptr(out["newton"]), _ptr(out["status"]), _stream(stream)))
    return out


def _autograd():
    import torch

    class HopfFn(torch.autograd.Function):
        """phi(x, t; A) with the hand-written envelope-theorem backward
        (hopf_backward): dphi/dx = v*, dphi/dt = -H(v*), dphi/dA = -1/2 v* v*^T.
        ``A_param`` is the tensor the caller differentiates with respect to
        (n x n, or n for a diagonal A); ``hopf`` must be a handle built from
        its current value.  Returns phi (float64, one per query); the gradient
        v* is available as ``hopf.last_grad``.  Second derivatives are not
        provided."""

        @staticmethod
        def forward(ctx, x, t, A_param, hopf):
            out = hopf.eval(x, t)
            hopf.last_grad = out["grad"]
            ctx.hopf = hopf
            ctx.save_for_backward(out["grad"])
            return out["phi"]

        @staticmethod
        def backward(ctx, g_phi):
            (vstar,) = ctx.saved_tensors
            need_x, need_t, need_A = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
            gx, gt, gA = ctx.hopf.backward(g_phi.contiguous().to(torch.float32), vstar, need_x, need_t, need_A)
            return gx, gt, gA, None

    return HopfFn


_HopfFn = None


def HopfFn():
    """The torch.autograd.Function class (created on first use)."""
    global _HopfFn
    if _HopfFn is None:
        _HopfFn = _autograd()
    return _HopfFn
