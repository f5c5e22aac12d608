"""Thin ctypes binding of libpmat (include/pmat.h): argument marshalling only.

Every step of every operation runs in the library's CUDA kernels; this module
only passes device pointers, sizes and the CUDA stream.  PyTorch provides
device memory and streams.  There is no CPU fallback: when libpmat.so is
missing or no GPU is present, calls raise.

Polynomial matrices are torch CUDA tensors of shape (rows, cols, length),
contiguous, with dtype uint32/int32 (w = 4) or uint64/int64 (w = 8); the
bits are read as unsigned residues in [0, p).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmat.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pmat.h")

PM_OK, PM_EINVAL, PM_EDOMAIN, PM_ENOMEM, PM_ECUDA, PM_ETIMEOUT, PM_EUNSUPPORTED, PM_ESCRATCH = range(8)
(PM_OPT_POINTWISE, PM_OPT_THRESHOLD, PM_OPT_DEBUG_CHECKS, PM_OPT_STAGE_TIMING, PM_OPT_LEAF_CLUSTER,
 PM_OPT_HOST_CHUNKS, PM_OPT_TEST_WITHHOLD_MMA) = 1, 2, 3, 4, 5, 6, 7
PM_NSTAGES = 8
STAGES = ["fwd_ntt", "pointwise", "inv_ntt", "crt", "leaf", "other"]
STATUS_NAMES = {0: "PM_OK", 1: "PM_EINVAL", 2: "PM_EDOMAIN", 3: "PM_ENOMEM", 4: "PM_ECUDA",
                5: "PM_ETIMEOUT", 6: "PM_EUNSUPPORTED", 7: "PM_ESCRATCH"}


class PmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class pmat_desc(C.Structure):
    _fields_ = [("p", C.c_uint64), ("w", C.c_int), ("m", C.c_int), ("n", C.c_int), ("k", C.c_int),
                ("A", C.c_void_p), ("dA", C.c_int64), ("B", C.c_void_p), ("dB", C.c_int64), ("C", C.c_void_p)]


_lib = None


def lib():
    """Load libpmat.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, i32, i64, u64 = C.c_void_p, C.c_int, C.c_int64, C.c_uint64
        sig = {
            "pm_create": ([C.POINTER(C.c_void_p), i32, P], i32),
            "pm_destroy": ([P], i32),
            "pm_set_option": ([P, i32, i64], i32),
            "pm_set_stream": ([P, P], i32),
            "pm_sync": ([P], i32),
            "pm_last_error": ([P], C.c_char_p),
            "pm_kernel_launches": ([P], i64),
            "pm_stage_times": ([P, P, P], i32),
            "pmat_mul": ([P, u64, i32, i32, i32, i32, P, i64, P, i64, P], i32),
            "pmat_mul_host": ([P, u64, i32, i32, i32, i32, P, i64, P, i64, P], i32),
            "pmat_mul_trunc": ([P, u64, i32, i32, i32, i32, P, i64, P, i64, i64, P], i32),
            "pmat_middle_product": ([P, u64, i32, i32, i32, i32, P, i64, P, i64, i64, i64, P], i32),
            "pmat_mul_batched": ([P, i32, C.POINTER(pmat_desc)], i32),
            "pmat_mul_noalloc": ([u64, i32, i32, i32, i32, P, i64, P, i64, P, P], i32),
            "pm_basis": ([P, u64, i32, i32, P, i64, i64, P, P, P], i32),
            "pm_intbasis": ([P, u64, i32, i32, P, i64, u64, u64, P, P, P], i32),
            "pmat_solve": ([P, u64, i32, P, i64, P, i64, P, P, P], i32),
            "pm_work_counters": ([P, P, i32], i32),
            "pm_host_join": ([P], i32),
            "bivariate_resultant_villard": ([P, i32, P, i32, i32, P, i32, i32, P, i32, P], i32),
            "bivariate_resultant": ([P, i32, P, i32, i32, P, i32, i32, P, P], i32),
            "pmat_inv_trunc": ([P, u64, i32, i32, P, i64, i64, P], i32),
            "pmat_solve_series": ([P, u64, i32, i32, P, i64, P, i64, i64, P], i32),
            "pmat_solve_series_hol": ([P, u64, i32, i32, P, i64, P, i64, i64, P], i32),
            "pmat_inv_slices": ([P, u64, i32, i32, P, i64, i32, P], i32),
            "pm_mma_rate": ([i32, i32, i32, C.POINTER(C.c_double)], i32),
            "pmat_mul_vdm": ([P, u64, i32, i32, i32, P, i64, P, i64, P], i32),
            "pm_tune_product": ([P, u64, i32, i32, i32, i32, i64, i64, i32, P], i32),
            "pm_tune_basis": ([P, u64, i32, i32, i64, i32, P], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def header_functions():
    """Names of the functions declared in include/pmat.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)) - {"if"})


# ------------------------------------------------------------------ helpers
def width(t: torch.Tensor) -> int:
    if t.dtype in (torch.int32, torch.uint32):
        return 4
    if t.dtype in (torch.int64, torch.uint64):
        return 8
    raise TypeError(f"unsupported dtype {t.dtype}")


def _dev(t: torch.Tensor) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t


def to_device(a: np.ndarray, device="cuda") -> torch.Tensor:
    """Copy a uint32/uint64 NumPy array to the device (stored as int32/int64 bits)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).to(device)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).to(device)
    raise TypeError(f"unsupported dtype {a.dtype}")


def to_host(t: torch.Tensor) -> np.ndarray:
    a = t.detach().cpu().contiguous().numpy()
    if a.dtype in (np.int64, np.uint64):
        return a.view(np.uint64)
    return a.view(np.uint32)


class Context:
    """One pm_ctx bound to a CUDA device and stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        L = lib()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        # handle 0 is torch's legacy default stream: pass cudaStreamLegacy (0x1),
        # since NULL asks the library for a stream of its own
        rc = L.pm_create(C.byref(h), device, C.c_void_p(stream.cuda_stream or 1))
        if rc != PM_OK:
            raise PmError(rc, "pm_create failed")
        self.h = h

    def _ck(self, rc: int):
        if rc != PM_OK:
            raise PmError(rc, lib().pm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().pm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: int, value: int):
        self._ck(lib().pm_set_option(self.h, key, value))

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._ck(lib().pm_set_stream(self.h, C.c_void_p(stream.cuda_stream or 1)))

    def sync(self):
        self._ck(lib().pm_sync(self.h))

    def launches(self) -> int:
        return int(lib().pm_kernel_launches(self.h))

    def host_join(self):
        """Make the context's stream wait for the downloads of earlier pmat_mul_host calls."""
        self._ck(lib().pm_host_join(self.h))

    def work(self, reset: bool = False):
        """{"bytes", "macs", "butterflies"}: algorithmic work of the products run so far."""
        out = np.zeros(3, dtype=np.int64)
        self._ck(lib().pm_work_counters(self.h, out.ctypes.data, 1 if reset else 0))
        return {"bytes": int(out[0]), "macs": int(out[1]), "butterflies": int(out[2])}

    def stage_times(self):
        """{stage: (ms, launches)} recorded since the last call (needs PM_OPT_STAGE_TIMING)."""
        ms = np.zeros(PM_NSTAGES, dtype=np.float64)
        nl = np.zeros(PM_NSTAGES, dtype=np.int64)
        self._ck(lib().pm_stage_times(self.h, ms.ctypes.data, nl.ctypes.data))
        return {name: (float(ms[i]), int(nl[i])) for i, name in enumerate(STAGES)}


def _out(out, shape, like):
    if out is None:
        return torch.empty(shape, dtype=like.dtype, device=like.device)
    if tuple(out.shape) != tuple(shape) or out.dtype != like.dtype:
        raise ValueError(f"out must be {shape} of {like.dtype}")
    return _dev(out)


def pmat_mul(ctx: Context, p: int, A: torch.Tensor, B: torch.Tensor, out=None) -> torch.Tensor:
    """C = A . B mod p (A: m x n x dA, B: n x k x dB) -> m x k x (dA + dB - 1)."""
    A, B = _dev(A), _dev(B)
    m, n, dA = A.shape
    n2, k, dB = B.shape
    if n != n2 or A.dtype != B.dtype:
        raise ValueError("shape/dtype mismatch")
    Cout = _out(out, (m, k, dA + dB - 1), A)
    ctx._ck(lib().pmat_mul(ctx.h, p, width(A), m, n, k, A.data_ptr(), dA, B.data_ptr(), dB, Cout.data_ptr()))
    return Cout


def _host(t: torch.Tensor) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("expected a CPU tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t


def pmat_mul_host(ctx: Context, p: int, A: torch.Tensor, B: torch.Tensor, out=None) -> torch.Tensor:
    """C = A . B mod p with A, B and C in host memory (pinned for overlap); asynchronous, and
    consecutive calls overlap: read C after ctx.sync()."""
    A, B = _host(A), _host(B)
    m, n, dA = A.shape
    n2, k, dB = B.shape
    if n != n2 or A.dtype != B.dtype:
        raise ValueError("shape/dtype mismatch")
    shape = (m, k, dA + dB - 1)
    if out is None:
        Cout = torch.empty(shape, dtype=A.dtype, pin_memory=A.is_pinned())
    else:
        if tuple(out.shape) != shape or out.dtype != A.dtype:
            raise ValueError(f"out must be {shape} of {A.dtype}")
        Cout = _host(out)
    ctx._ck(lib().pmat_mul_host(ctx.h, p, width(A), m, n, k, A.data_ptr(), dA, B.data_ptr(), dB, Cout.data_ptr()))
    return Cout


def pmat_mul_trunc(ctx: Context, p: int, A, B, t: int, out=None) -> torch.Tensor:
    """C = A . B mod x^t -> m x k x t."""
    A, B = _dev(A), _dev(B)
    m, n, dA = A.shape
    _, k, dB = B.shape
    Cout = _out(out, (m, k, t), A)
    ctx._ck(lib().pmat_mul_trunc(ctx.h, p, width(A), m, n, k, A.data_ptr(), dA, B.data_ptr(), dB, t,
                                 Cout.data_ptr()))
    return Cout


def pmat_inv_trunc(ctx: Context, p: int, A, t: int, out=None) -> torch.Tensor:
    """X = A^-1 mod x^t -> n x n x t (A: n x n x dA with A(0) invertible mod the prime p).

    A singular A(0) is reported by the next ctx.sync() (PM_EDOMAIN)."""
    A = _dev(A)
    n, n2, dA = A.shape
    if n != n2:
        raise ValueError("A must be square")
    X = _out(out, (n, n, t), A)
    ctx._ck(lib().pmat_inv_trunc(ctx.h, p, width(A), n, A.data_ptr(), dA, t, X.data_ptr()))
    return X


def pmat_solve_series(ctx: Context, p: int, A, b, N: int, out=None) -> torch.Tensor:
    """v = A^-1 b mod x^N -> n x 1 x N (A: n x n x dA with A(0) invertible mod the prime p,
    b: n x 1 x db, same width).  A singular A(0) is reported by the next ctx.sync() (PM_EDOMAIN)."""
    A, b = _dev(A), _dev(b)
    n, n2, dA = A.shape
    if n != n2 or b.shape[0] != n or b.shape[1] != 1 or b.dtype != A.dtype:
        raise ValueError("A must be n x n and b n x 1 of the same width")
    v = _out(out, (n, 1, N), A)
    ctx._ck(lib().pmat_solve_series(ctx.h, p, width(A), n, A.data_ptr(), dA, b.data_ptr(), b.shape[2], N,
                                    v.data_ptr()))
    return v


def pmat_solve_series_hol(ctx: Context, p: int, A, b, N: int, out=None) -> torch.Tensor:
    """v = A^-1 b mod x^N by high-order lifting (the same result as pmat_solve_series): needs
    dA >= 2, db <= dA and N within 256 residues of degree dA - 1."""
    A, b = _dev(A), _dev(b)
    n, n2, dA = A.shape
    if n != n2 or b.shape[0] != n or b.shape[1] != 1 or b.dtype != A.dtype:
        raise ValueError("A must be n x n and b n x 1 of the same width")
    v = _out(out, (n, 1, N), A)
    ctx._ck(lib().pmat_solve_series_hol(ctx.h, p, width(A), n, A.data_ptr(), dA, b.data_ptr(), b.shape[2], N,
                                        v.data_ptr()))
    return v


def pmat_inv_slices(ctx: Context, p: int, A, K: int, out=None) -> torch.Tensor:
    """High-order lifting slices -> K x n x n x (2D+1): slice i = coefficients (2^i - 1) D ..
    (2^i + 1) D of A^-1 (A: n x n x dA, D = dA - 1, A(0) invertible mod the prime p)."""
    A = _dev(A)
    n, n2, dA = A.shape
    if n != n2:
        raise ValueError("A must be square")
    S = _out(out, (K, n, n, 2 * (dA - 1) + 1), A)
    ctx._ck(lib().pmat_inv_slices(ctx.h, p, width(A), n, A.data_ptr(), dA, K, S.data_ptr()))
    return S


def pmat_middle_product(ctx: Context, p: int, A, B, c: int, d: int, out=None) -> torch.Tensor:
    """Coefficients c .. c+d-1 of A . B -> m x k x d."""
    A, B = _dev(A), _dev(B)
    m, n, dA = A.shape
    _, k, dB = B.shape
    Cout = _out(out, (m, k, d), A)
    ctx._ck(lib().pmat_middle_product(ctx.h, p, width(A), m, n, k, A.data_ptr(), dA, B.data_ptr(), dB, c, d,
                                      Cout.data_ptr()))
    return Cout


def pmat_mul_batched(ctx: Context, items, outs=None):
    """items: list of (p, A, B); returns the list of products (each as pmat_mul)."""
    n = len(items)
    arr = (pmat_desc * max(n, 1))()
    res = []
    for i, (p, A, B) in enumerate(items):
        A, B = _dev(A), _dev(B)
        m, nn, dA = A.shape
        _, k, dB = B.shape
        Cout = _out(outs[i] if outs else None, (m, k, dA + dB - 1), A)
        arr[i] = pmat_desc(p, width(A), m, nn, k, A.data_ptr(), dA, B.data_ptr(), dB, Cout.data_ptr())
        res.append(Cout)
    ctx._ck(lib().pmat_mul_batched(ctx.h, n, arr))
    return res


def pm_basis(ctx: Context, p: int, F: torch.Tensor, d: int, shift, out=None):
    """PM-Basis (Algorithm 3): returns (P as m x m x (d+1) uint64 bits, rdeg_s(P) as int64 array)."""
    F = _dev(F)
    if width(F) != 8:
        raise TypeError("pm_basis takes 64-bit coefficients")
    m, n, lenF = F.shape
    s = np.ascontiguousarray(np.asarray(shift, dtype=np.int64))
    if s.shape != (m,):
        raise ValueError("shift must have m entries")
    P = _out(out, (m, m, d + 1), F)
    rd = np.zeros(m, dtype=np.int64)
    ctx._ck(lib().pm_basis(ctx.h, p, m, n, F.data_ptr(), lenF, d, s.ctypes.data, P.data_ptr(), rd.ctypes.data))
    return P, rd


def pmat_solve(ctx: Context, p: int, A: torch.Tensor, b: torch.Tensor):
    """Lifting solver (Sec. 4): (u, f, deg f, deg u) with A u = f b, f monic of minimal degree.
    A: n x n x dA, b: n x 1 x db (64-bit); u: n x 1 x (D2+1), f: D1+1 (device tensors)."""
    A, b = _dev(A), _dev(b)
    if width(A) != 8 or width(b) != 8:
        raise TypeError("pmat_solve takes 64-bit coefficients")
    n, n2, dA = A.shape
    if n != n2 or tuple(b.shape[:2]) != (n, 1):
        raise ValueError("A must be n x n and b n x 1")
    db = b.shape[2]
    D1 = n * (dA - 1)
    D2 = (n - 1) * (dA - 1) + db - 1
    u = torch.empty((n, 1, D2 + 1), dtype=A.dtype, device=A.device)
    f = torch.empty((D1 + 1,), dtype=A.dtype, device=A.device)
    dg = np.zeros(2, dtype=np.int64)
    ctx._ck(lib().pmat_solve(ctx.h, p, n, A.data_ptr(), dA, b.data_ptr(), db, u.data_ptr(), f.data_ptr(),
                             dg.ctypes.data))
    return u, f, int(dg[0]), int(dg[1])


def pm_intbasis(ctx: Context, p: int, E: torch.Tensor, c: int, q: int, shift, out=None):
    """PM-IntBasis (Algorithm 5) at the points c q^l: E is m x n x sigma (E[:, :, l] goes with
    c q^l); returns (P as m x m x (sigma+1) uint64 bits, rdeg_s(P) as int64 array)."""
    E = _dev(E)
    if width(E) != 8:
        raise TypeError("pm_intbasis takes 64-bit coefficients")
    m, n, sigma = E.shape
    s = np.ascontiguousarray(np.asarray(shift, dtype=np.int64))
    if s.shape != (m,):
        raise ValueError("shift must have m entries")
    P = _out(out, (m, m, sigma + 1), E)
    rd = np.zeros(m, dtype=np.int64)
    ctx._ck(lib().pm_intbasis(ctx.h, p, m, n, E.data_ptr(), sigma, c, q, s.ctypes.data, P.data_ptr(),
                              rd.ctypes.data))
    return P, rd


def bivariate_resultant_villard(ctx: Context, primes, f: torch.Tensor, g: torch.Tensor, m: int = 0,
                                out=None) -> torch.Tensor:
    """Res_y(f, g) modulo each prime by the variant of Algorithm 6 (Sec. 5.2); same layout as
    bivariate_resultant; m = 0 takes the default block size."""
    f, g = _dev(f), _dev(g)
    if f.dim() == 2:
        f, g = f.unsqueeze(0), g.unsqueeze(0)
    npr, dyf1, dxf1 = f.shape
    _, dyg1, dxg1 = g.shape
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64).reshape(-1))
    if len(pr) != npr:
        raise ValueError("one prime per instance")
    D = (dxf1 - 1) * (dyg1 - 1) + (dxg1 - 1) * (dyf1 - 1)
    R = _out(out, (npr, D + 1), f)
    ctx._ck(lib().bivariate_resultant_villard(ctx.h, npr, pr.ctypes.data, dxf1 - 1, dyf1 - 1, f.data_ptr(),
                                              dxg1 - 1, dyg1 - 1, g.data_ptr(), m, R.data_ptr()))
    return R


def bivariate_resultant(ctx: Context, primes, f: torch.Tensor, g: torch.Tensor, out=None) -> torch.Tensor:
    """Res_y(f, g) modulo each prime.  f: (nprimes, dyf+1, dxf+1) 64-bit, f[., j, i] = coeff of x^i y^j."""
    f, g = _dev(f), _dev(g)
    if f.dim() == 2:
        f, g = f.unsqueeze(0), g.unsqueeze(0)
    npr, dyf1, dxf1 = f.shape
    _, dyg1, dxg1 = g.shape
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64).reshape(-1))
    if len(pr) != npr:
        raise ValueError("one prime per instance")
    D = (dxf1 - 1) * (dyg1 - 1) + (dxg1 - 1) * (dyf1 - 1)
    R = _out(out, (npr, D + 1), f)
    ctx._ck(lib().bivariate_resultant(ctx.h, npr, pr.ctypes.data, dxf1 - 1, dyf1 - 1, f.data_ptr(), dxg1 - 1,
                                      dyg1 - 1, g.data_ptr(), R.data_ptr()))
    return R


def mma_rate(device: int = 0, n_cols: int = 256, iters: int = 4096) -> float:
    """Measured TFLOP/s of dense tcgen05.mma kind::f16 (M = 128, N = n_cols, K = 16) on one GPU."""
    out = C.c_double(0.0)
    rc = lib().pm_mma_rate(device, n_cols, iters, C.byref(out))
    if rc != PM_OK:
        raise PmError(rc, "pm_mma_rate failed")
    return out.value


def tune_product(ctx: Context, p: int, w: int, m: int, n: int, k: int, dA: int, dB: int, reps: int = 3):
    """pm_tune_product: (form, bi, bk, pointwise ns per product, candidates timed)."""
    out = np.zeros(5, dtype=np.int64)
    ctx._ck(lib().pm_tune_product(ctx.h, p, w, m, n, k, dA, dB, reps, out.ctypes.data))
    return tuple(int(v) for v in out)


def tune_basis(ctx: Context, p: int, m: int, n: int, d: int, reps: int = 1):
    """pm_tune_basis: (threshold T, ns per call); the context's threshold is set to T."""
    out = np.zeros(2, dtype=np.int64)
    ctx._ck(lib().pm_tune_basis(ctx.h, p, m, n, d, reps, out.ctypes.data))
    return tuple(int(v) for v in out)


def pmat_mul_vdm(ctx: Context, p: int, A: torch.Tensor, B: torch.Tensor, out=None):
    """pmat_mul by Vandermonde-matrix evaluation / interpolation on the tensor cores (uint32, NTT prime p)."""
    A, B = _dev(A), _dev(B)
    if width(A) != 4 or width(B) != 4:
        raise TypeError("pmat_mul_vdm takes 32-bit coefficients")
    m, n, dA = A.shape
    n2, k, dB = B.shape
    if n2 != n:
        raise ValueError("inner dimensions differ")
    C = _out(out, (m, k, dA + dB - 1), A)
    ctx._ck(lib().pmat_mul_vdm(ctx.h, p, m, n, k, A.data_ptr(), dA, B.data_ptr(), dB, C.data_ptr()))
    return C

