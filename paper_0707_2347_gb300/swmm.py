"""Python binding of the C ABI in include/swmm.h (ctypes; marshalling only).

Every step of the computation runs in the library's CUDA kernels; this
module only turns torch tensors into (device pointer, leading dimension)
pairs, passes the current torch CUDA stream, and checks return codes.
Loading fails loudly when the shared library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libswmm.so")

# return codes
OK, EINVAL, ENOMEM, EUNSUPPORTED, ECUDA, ETIMEOUT = range(6)
HOOK_WAIT_NS, HOOK_STALL_GEMMS, HOOK_FAIL_ALLOCS, HOOK_LOWMEM_BYTES = 1, 2, 3, 4  # swmm_test_hook
# modes
MODP, FP32 = 0, 1
# schedules (paper table numbers)
CLASSICAL, T1_DHSS, T2_HLJJTT, T3_IP, T4_OVL, T5_OVR = 0, 1, 2, 3, 4, 5
T6_ACLR, T7_ACCR, T8_ACR, T9_ACC, IPMM, T4M_OVL, IP0VMM, TBLOCK, CUSTOM = 6, 7, 8, 9, 10, 11, 12, 13, 14
AUTO = -1
SCHED_NAMES = {CLASSICAL: "classical", T1_DHSS: "T1", T2_HLJJTT: "T2", T3_IP: "IP", T4_OVL: "OvL",
               T5_OVR: "OvR", T6_ACLR: "AcLR", T7_ACCR: "AccR", T8_ACR: "AcR", T9_ACC: "Acc",
               IPMM: "IPMM", T4M_OVL: "OvLM", IP0VMM: "IP0vMM", TBLOCK: "Sec7.2", CUSTOM: "custom"}
# flags
FLAG_UNFUSED, FLAG_SIMT_LEAF, FLAG_TIMING, FLAG_GRAPH, FLAG_SERIAL, FLAG_LOWMEM, FLAG_TUNE = 1, 2, 4, 8, 16, 32, 64
LOWMEM_STAGE_BYTES = 64 << 20


class SwmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"swmm error {code}: {msg}")
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("p", ctypes.c_uint32), ("sched", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("flags", ctypes.c_uint32), ("ipmm_cutoff", ctypes.c_int32),
                ("ipmm_acc", ctypes.c_int32), ("tblock", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("workspace_bytes", ctypes.c_int64), ("plan_extra_elems", ctypes.c_int64),
                ("paper_extra_elems", ctypes.c_int64), ("add_elems", ctypes.c_int64),
                ("leaf_flops", ctypes.c_int64), ("leaf_launches", ctypes.c_int64),
                ("ew_launches", ctypes.c_int64), ("leaf_products", ctypes.c_int64),
                ("staging_bytes", ctypes.c_int64), ("pack_bytes", ctypes.c_int64),
                ("level_packs", ctypes.c_int64), ("reserved", ctypes.c_int64 * 5)]


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("k", ctypes.c_int64), ("n", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64), ("mode", ctypes.c_int32), ("p", ctypes.c_uint32),
                ("alpha_u", ctypes.c_uint32), ("beta_u", ctypes.c_uint32), ("alpha_f", ctypes.c_float),
                ("beta_f", ctypes.c_float), ("sched", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("chosen_sched", ctypes.c_int32), ("chosen_depth", ctypes.c_int32)]


# every symbol include/swmm.h declares
EXPORTS = ["swmm_create", "swmm_destroy", "swmm_set_stream", "swmm_mul", "swmm_muladd", "swmm_muladd_noalloc",
           "swmm_mul_inplace",
           "swmm_muladd_batched", "swmm_autotune", "swmm_workspace_elems", "swmm_leaf_timing", "swmm_get_stats",
           "swmm_sync", "swmm_strerror", "swmm_last_error", "swmm_matvec", "swmm_residual", "swmm_muladd_host",
           "swmm_test_hook", "swmm_memory_use", "swmm_plan_stats",
           # include/swmm_search.h (host only, see search.py)
           "swmm_schedule_search", "swmm_schedule_check", "swmm_search_node_name", "swmm_search_node_count",
           "swmm_set_schedule", "swmm_schedule_workspace", "swmm_schedule_stats", "swmm_table_rows"]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libswmm.so (no GPU needed).  Raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    i64, vp, cvp = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
    lib.swmm_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
    lib.swmm_destroy.argtypes = [vp]
    lib.swmm_set_stream.argtypes = [vp, vp]
    lib.swmm_mul.argtypes = [vp, i64, i64, i64, cvp, i64, cvp, i64, vp, i64, ctypes.POINTER(_Opts)]
    lib.swmm_muladd.argtypes = [vp, i64, i64, i64, cvp, cvp, i64, cvp, i64, cvp, vp, i64, ctypes.POINTER(_Opts)]
    lib.swmm_muladd_noalloc.argtypes = [vp, i64, i64, i64, cvp, cvp, i64, cvp, i64, cvp, vp, i64,
                                        ctypes.POINTER(_Opts)]
    lib.swmm_mul_inplace.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64, vp, i64, cvp, cvp,
                                     ctypes.POINTER(_Opts)]
    lib.swmm_workspace_elems.argtypes = [vp, i64, i64, i64, ctypes.POINTER(_Opts), ctypes.POINTER(i64),
                                         ctypes.POINTER(i64)]
    lib.swmm_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    lib.swmm_muladd_batched.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_uint32]
    lib.swmm_autotune.argtypes = [vp, i64, i64, i64, ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(i64)]
    lib.swmm_leaf_timing.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.swmm_sync.argtypes = [vp]
    lib.swmm_test_hook.argtypes = [vp, ctypes.c_int32, i64]
    lib.swmm_memory_use.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i64)]
    lib.swmm_matvec.argtypes = [vp, i64, i64, cvp, i64, cvp, vp, ctypes.POINTER(_Opts)]
    lib.swmm_muladd_host.argtypes = [vp, i64, i64, i64, cvp, cvp, i64, cvp, i64, cvp, vp, i64,
                                     ctypes.POINTER(_Opts)]
    lib.swmm_residual.argtypes = [vp, i64, i64, i64, cvp, cvp, i64, cvp, i64, cvp, cvp, cvp, i64, cvp, vp,
                                  ctypes.POINTER(_Opts)]
    lib.swmm_strerror.argtypes = [ctypes.c_int]
    lib.swmm_strerror.restype = ctypes.c_char_p
    lib.swmm_last_error.argtypes = [vp]
    lib.swmm_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
    lib.swmm_strerror.restype = ctypes.c_char_p
    lib.swmm_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


@dataclass
class Opts:
    mode: int = MODP
    p: int = 65521
    sched: int = T9_ACC
    depth: int = 1
    flags: int = 0
    ipmm_cutoff: int = 0
    ipmm_acc: int = 0
    tblock: int = 0

    def c(self) -> _Opts:
        return _Opts(self.mode, self.p, self.sched, self.depth, self.flags, self.ipmm_cutoff, self.ipmm_acc,
                     self.tblock)


def autotune(m, k, n, mode=MODP, p=65521):
    """(sched, depth, modelled microseconds, peak temporary elements) the
    library's autotuner picks; no GPU needed."""
    lib = load()
    s, d = ctypes.c_int32(), ctypes.c_int32()
    t, e = ctypes.c_double(), ctypes.c_int64()
    rc = lib.swmm_autotune(None, m, k, n, mode, p, ctypes.byref(s), ctypes.byref(d), ctypes.byref(t), ctypes.byref(e))
    if rc != OK:
        raise SwmmError(rc, "autotune failed")
    return s.value, d.value, t.value, e.value


def plan_stats(m, k, n, opts) -> dict:
    """The counts of the plan an eager call with these sizes and options
    would run (swmm_plan_stats); no GPU needed."""
    lib = load()
    st = _Stats()
    rc = lib.swmm_plan_stats(None, m, k, n, ctypes.byref(opts.c()), ctypes.byref(st))
    if rc != OK:
        raise SwmmError(rc, "planning failed")
    return {f: getattr(st, f) for f, _ in _Stats._fields_ if f != "reserved"}


def _scalar(mode, v):
    if v is None:
        return None
    if mode == MODP:
        return ctypes.byref(ctypes.c_uint32(int(v) & 0xFFFFFFFF))
    return ctypes.byref(ctypes.c_float(float(v)))


def _mat(t, what):
    """(device pointer, ld) of a 2-D row-major torch tensor."""
    if t is None:
        return None, 1
    if t.dim() != 2 or (t.shape[1] > 1 and t.stride(1) != 1):
        raise ValueError(f"{what} must be a 2-D row-major tensor")
    return ctypes.c_void_p(t.data_ptr()), max(int(t.stride(0)), int(t.shape[1]), 1)


def _vec(t):
    """device pointer of a contiguous 1-D tensor (None -> NULL)."""
    if t is None:
        return None
    if t.dim() != 1 or (t.numel() > 1 and t.stride(0) != 1):
        raise ValueError("vectors must be contiguous 1-D tensors")
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """One library handle on one CUDA device.  Calls run asynchronously on
    the current torch CUDA stream."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.h = ctypes.c_void_p()
        rc = self.lib.swmm_create(ctypes.byref(self.h), int(device), None)
        if rc != OK:
            raise SwmmError(rc, "swmm_create failed")
        self.device = device

    def close(self):
        if self.h:
            self.lib.swmm_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        import torch
        s = torch.cuda.current_stream(self.device).cuda_stream
        self.lib.swmm_set_stream(self.h, ctypes.c_void_p(s))

    def _check(self, rc):
        if rc != OK:
            msg = self.lib.swmm_last_error(self.h).decode() or self.lib.swmm_strerror(rc).decode()
            raise SwmmError(rc, msg)

    def mul(self, A, B, C, opts: Opts):
        """C <- A B (read-only A, B)."""
        self._stream()
        a, lda = _mat(A, "A")
        b, ldb = _mat(B, "B")
        c, ldc = _mat(C, "C")
        m, k = A.shape
        n = B.shape[1]
        self._check(self.lib.swmm_mul(self.h, m, k, n, a, lda, b, ldb, c, ldc, ctypes.byref(opts.c())))
        return C

    def muladd(self, alpha, A, B, beta, C, opts: Opts):
        """C <- alpha A B + beta C (read-only A, B)."""
        self._stream()
        a, lda = _mat(A, "A")
        b, ldb = _mat(B, "B")
        c, ldc = _mat(C, "C")
        m, k = A.shape
        n = B.shape[1]
        self._check(self.lib.swmm_muladd(self.h, m, k, n, _scalar(opts.mode, alpha), a, lda, b, ldb,
                                         _scalar(opts.mode, beta), c, ldc, ctypes.byref(opts.c())))
        return C

    def muladd_noalloc(self, alpha, A, B, beta, C, opts: Opts):
        """swmm_muladd_noalloc: like muladd, scratch from the library's static
        device array (no allocation)."""
        self._stream()
        a, lda = _mat(A, "A")
        b, ldb = _mat(B, "B")
        c, ldc = _mat(C, "C")
        m, k = A.shape
        n = B.shape[1]
        self._check(self.lib.swmm_muladd_noalloc(self.h, m, k, n, _scalar(opts.mode, alpha), a, lda, b, ldb,
                                                 _scalar(opts.mode, beta), c, ldc, ctypes.byref(opts.c())))
        return C

    def muladd_host(self, alpha, A, B, beta, C, opts: Opts):
        """swmm_muladd_host: C <- alpha A B + beta C with A, B, C host (CPU)
        tensors, page-locked for overlap; C holds the result after sync()."""
        self._stream()
        for t, what in ((A, "A"), (B, "B"), (C, "C")):
            if t.is_cuda:
                raise ValueError(f"{what} must be a host tensor")
        a, lda = _mat(A, "A")
        b, ldb = _mat(B, "B")
        c, ldc = _mat(C, "C")
        m, k = A.shape
        n = B.shape[1]
        self._check(self.lib.swmm_muladd_host(self.h, m, k, n, _scalar(opts.mode, alpha), a, lda, b, ldb,
                                              _scalar(opts.mode, beta), c, ldc, ctypes.byref(opts.c())))
        return C

    def matvec(self, M, x, y, opts: Opts):
        """swmm_matvec: y = M x (mod p: uint32 x, y as int32 tensors holding
        [0, p); FP32 mode: float64 x, y)."""
        self._stream()
        mp, ldm = _mat(M, "M")
        rows, cols = M.shape
        self._check(self.lib.swmm_matvec(self.h, rows, cols, mp, ldm, _vec(x), _vec(y), ctypes.byref(opts.c())))
        return y

    def residual(self, alpha, A, B, beta, y0, C, x, r, opts: Opts):
        """swmm_residual: r = C x - alpha A (B x) - beta y0 with y0 = C_in x
        (None when beta is 0)."""
        self._stream()
        a, lda = _mat(A, "A")
        b, ldb = _mat(B, "B")
        c, ldc = _mat(C, "C")
        m, k = A.shape
        n = B.shape[1]
        self._check(self.lib.swmm_residual(self.h, m, k, n, _scalar(opts.mode, alpha), a, lda, b, ldb,
                                           _scalar(opts.mode, beta), _vec(y0), c, ldc, _vec(x), _vec(r),
                                           ctypes.byref(opts.c())))
        return r

    def mul_inplace(self, A, B, C, opts: Opts, alpha=1, beta=None):
        """Schedules that may overwrite A and/or B (Tables 3-8)."""
        self._stream()
        a, lda = _mat(A, "A")
        b, ldb = _mat(B, "B")
        c, ldc = _mat(C, "C")
        m, k = A.shape
        n = B.shape[1]
        self._check(self.lib.swmm_mul_inplace(self.h, m, k, n, a, lda, b, ldb, c, ldc, _scalar(opts.mode, alpha),
                                              _scalar(opts.mode, beta), ctypes.byref(opts.c())))
        return C

    def muladd_batched(self, problems, flags: int = 0):
        """problems: list of dicts with A, B, C (torch tensors), mode, p,
        alpha, beta, sched (AUTO default), depth.  Returns the (sched, depth)
        each problem ran with."""
        self._stream()
        arr = (Problem * len(problems))()
        for i, q in enumerate(problems):
            a, lda = _mat(q["A"], "A")
            b, ldb = _mat(q["B"], "B")
            c, ldc = _mat(q["C"], "C")
            mode = q.get("mode", MODP)
            arr[i] = Problem(q["A"].shape[0], q["A"].shape[1], q["B"].shape[1], a, lda, b, ldb, c, ldc, mode,
                             q.get("p", 65521), int(q.get("alpha", 1)) if mode == MODP else 0,
                             int(q.get("beta", 1)) if mode == MODP else 0,
                             float(q.get("alpha", 1.0)) if mode == FP32 else 0.0,
                             float(q.get("beta", 1.0)) if mode == FP32 else 0.0,
                             q.get("sched", AUTO), q.get("depth", 0), 0, 0)
        self._check(self.lib.swmm_muladd_batched(self.h, len(problems), arr, flags))
        return [(arr[i].chosen_sched, arr[i].chosen_depth) for i in range(len(problems))]

    def workspace_elems(self, m, k, n, opts: Opts):
        paper = ctypes.c_int64()
        plan = ctypes.c_int64()
        self._check(self.lib.swmm_workspace_elems(self.h, m, k, n, ctypes.byref(opts.c()), ctypes.byref(paper),
                                                  ctypes.byref(plan)))
        return paper.value, plan.value

    def stats(self) -> dict:
        s = _Stats()
        self._check(self.lib.swmm_get_stats(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _Stats._fields_ if f != "reserved"}

    def leaf_timing(self, reset: bool = True):
        """(gemm_ms, launches, tensor_flops) of leaf GEMM launches made with
        FLAG_TIMING since the last reset (waits for the stream)."""
        ms, n, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.swmm_leaf_timing(self.h, 1 if reset else 0, ctypes.byref(ms), ctypes.byref(n),
                                              ctypes.byref(fl)))
        return ms.value, n.value, fl.value

    def sync(self):
        self._check(self.lib.swmm_sync(self.h))

    def memory_use(self, reset: bool = False):
        """(pool_current, pool_high, graph_current, graph_high) in bytes
        (swmm_memory_use); reset sets both high-water marks to the current use."""
        out = (ctypes.c_int64 * 4)()
        self._check(self.lib.swmm_memory_use(self.h, 1 if reset else 0, out))
        return tuple(out)

    def measure_peak(self):
        """Context manager: .peak = the largest rise of device memory (default
        pool or graph memory) above its use at entry, while inside."""
        handle = self

        class _Peak:
            def __enter__(self):
                self.start = handle.memory_use(reset=True)
                return self

            def __exit__(self, *exc):
                if exc[0] is None:
                    end = handle.memory_use()
                    self.peak = max(end[1] - self.start[0], end[3] - self.start[2], 0)

        return _Peak()

    def test_hook(self, hook: int, value: int):
        """Failure injection for error-path tests (swmm_test_hook)."""
        self._check(self.lib.swmm_test_hook(self.h, hook, value))
