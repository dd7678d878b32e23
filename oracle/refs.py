"""Oracle: reference kernel outputs (test infrastructure only).

FP64 references follow the mathematical definition of each computation
(matmul, Section "Illustrative Example"; DG, Section "DG"; stencil, Section
"Finite Differences").  The calibration-suite kernels and the work-removed
twins have a fixed operation order, so the oracle replays them bit-exactly in
their own precision (compiled without multiply-add contraction).
"""
import ctypes

import numpy as np

from . import lib

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ready = False


def _setup():
    global _ready
    if _ready:
        return
    L = lib()
    L.oracle_stream_ref.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.c_void_p]
    L.oracle_fma_ref.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_void_p,
                                 ctypes.c_void_p]
    L.oracle_mm_ref.argtypes = [ctypes.c_longlong, _f32p, _f32p, _f64p, _f64p]
    L.oracle_dg_ref.argtypes = [ctypes.c_longlong, ctypes.c_longlong, _f32p, _f32p, _f64p, _f64p]
    L.oracle_fd_ref.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_double, ctypes.c_double, _f32p,
                                _f64p, _f64p]
    L.oracle_mm_twin_ref.argtypes = [ctypes.c_int, ctypes.c_longlong, _f32p, _f32p]
    L.oracle_dg_twin_ref.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
                                     ctypes.c_longlong, _f32p, _f32p, _f32p]
    L.oracle_fd_twin_ref.argtypes = [ctypes.c_int, ctypes.c_longlong, _f32p, _f32p]
    _u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
    L.oracle_mm_tc_ref.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, _u16p, _u16p, _f64p, _f64p]
    _ready = True


def stream(ins):
    """out[e] = ((in0[e] + in1[e]) + ...) in the inputs' dtype (fp32 or fp64)."""
    _setup()
    ins = [np.ascontiguousarray(x) for x in ins]
    dt = ins[0].dtype
    out = np.empty_like(ins[0])
    ptrs = (ctypes.c_void_p * len(ins))(*[x.ctypes.data for x in ins])
    lib().oracle_stream_ref(0 if dt == np.float32 else 1, len(ins), ins[0].size, ptrs, out.ctypes.data)
    return out


def fma(seed, op, F):
    """Arithmetic kernel output per work-item (op 0 add, 1 mul, 2 madd)."""
    _setup()
    seed = np.ascontiguousarray(seed)
    out = np.empty_like(seed)
    lib().oracle_fma_ref(0 if seed.dtype == np.float32 else 1, op, F, seed.size, seed.ctypes.data, out.ctypes.data)
    return out


def matmul(a, b):
    """FP64 C = A B and sum_k |a_ik b_kj|."""
    _setup()
    n = a.shape[0]
    c = np.empty((n, n)); ca = np.empty((n, n))
    lib().oracle_mm_ref(n, np.ascontiguousarray(a, np.float32), np.ascontiguousarray(b, np.float32), c, ca)
    return c, ca


def matmul_rows(a_rows, b):
    """FP64 rows of C = A B for the given rows of A (r x n) and all of B
    (n x n), with sum_k |a_ik b_kj|: the same definition as matmul, for
    sampled rows of a product too large to form whole (one FP64 matrix
    product per quantity)."""
    a64 = np.asarray(a_rows, dtype=np.float32).astype(np.float64)
    b64 = np.asarray(b, dtype=np.float32).astype(np.float64)
    return a64 @ b64, np.abs(a64) @ np.abs(b64)


def matmul_bf16_tn(a_bits, bt_bits):
    """FP64 C = A Bt^T over bf16 inputs given as uint16 bit patterns, and the |.| sums."""
    _setup()
    m, k = a_bits.shape
    n = bt_bits.shape[0]
    c = np.empty((m, n)); ca = np.empty((m, n))
    lib().oracle_mm_tc_ref(m, n, k, np.ascontiguousarray(a_bits, np.uint16), np.ascontiguousarray(bt_bits, np.uint16),
                           c, ca)
    return c, ca


def dg(D, u):
    """FP64 res[m,k,i] = sum_j D[m,i,j] u[k,j] and the |.| sums."""
    _setup()
    Np = D.shape[1]
    Nel = u.shape[0]
    res = np.empty((3, Nel, Np)); ra = np.empty((3, Nel, Np))
    lib().oracle_dg_ref(Np, Nel, np.ascontiguousarray(D, np.float32), np.ascontiguousarray(u, np.float32), res, ra)
    return res, ra


def stencil(u, c0, c1):
    """FP64 five-point stencil on the (n+2)x(n+2) input and the |.| sums."""
    return stencil_rows(u, c0, c1)


def stencil_rows(u, c0, c1):
    """FP64 five-point stencil on an (h+2) x (n+2) block of rows -> h x n."""
    _setup()
    h, n = u.shape[0] - 2, u.shape[1] - 2
    res = np.empty((h, n)); ra = np.empty((h, n))
    lib().oracle_fd_ref(h, n, c0, c1, np.ascontiguousarray(u, np.float32), res, ra)
    return res, ra


_MM_V = {"mm_pf_a": 2, "mm_pf_b": 3, "mm_nopf_a": 4, "mm_nopf_b": 5}
_DG_V = {"dg_nopf_u": 2, "dg_nopf_dm": 3, "dg_dmpf_u": 4, "dg_dmpf_dm": 5, "dg_upf_u": 9, "dg_dmpft_u": 10}
_FD_V = {"fd_tile_u": 2, "fd_direct_u": 4, "fd_tile18_u": 7}


def mm_twin(kernel, x):
    _setup()
    n = x.shape[0]
    dest = np.empty((n, n), np.float32)
    lib().oracle_mm_twin_ref(_MM_V[kernel], n, np.ascontiguousarray(x, np.float32), dest)
    return dest


def dg_twin(kernel, D, u, L0, L1):
    """Twin output in the kernel's own layout (dg_dmpft_u reads u as uT[j, k])."""
    _setup()
    Np = D.shape[1]
    Nel = u.shape[1] if kernel == "dg_dmpft_u" else u.shape[0]
    rows = -(-Np // L1) * L1
    dest = np.empty((rows, Nel), np.float32)
    lib().oracle_dg_twin_ref(_DG_V[kernel], Np, Nel, L0, L1, np.ascontiguousarray(D, np.float32),
                             np.ascontiguousarray(u, np.float32), dest)
    return dest


def fd_twin(kernel, u):
    _setup()
    n = u.shape[0] - 2
    G = -(-n // (14 if kernel == "fd_tile_u" else 16))
    T = 18 if kernel == "fd_tile18_u" else 16
    dest = np.empty((T * G, T * G), np.float32)
    lib().oracle_fd_twin_ref(_FD_V[kernel], n, np.ascontiguousarray(u, np.float32), dest)
    return dest
