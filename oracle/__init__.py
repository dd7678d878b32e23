"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_1904_09538_gb300``) and never imports
it; the only module both sides use is ``pm_inputs`` (seeded synthetic inputs,
no method arithmetic).

Contents
  enum.c        brute-force loop-domain enumeration (Algorithm 1, Algorithm 2)
                and FP64 / bit-exact reference kernel outputs (plain C)
  features.py   feature naming and model-feature matching (Section "Kernel
                Features", "Data Motion Features")
  model.py      model expressions: parse, evaluate, symbolic derivative
                (Section "Modeling Kernel Execution Time", "Computing Model
                Parameters")
  fit.py        linear and Levenberg-Marquardt calibration in FP64, geometric
                mean relative error (Section "Computing Model Parameters",
                "Results")
  quasipoly.py  exact interpolation of counts, which are quasi-polynomials in
                the size parameters (Section "Gathering Kernel Statistics")
"""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "enum.c")
_lib = None


def build(force=False):
    """Compile enum.c with gcc (no fused multiply-add contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Orec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("name", ctypes.c_char * 24), ("dtype", ctypes.c_char * 16),
                ("mem", ctypes.c_int), ("dir", ctypes.c_int), ("dsize", ctypes.c_int),
                ("uniform", ctypes.c_int), ("affine", ctypes.c_int),
                ("lstr", ctypes.c_longlong * 3), ("gstr", ctypes.c_longlong * 3), ("loopstr", ctypes.c_longlong),
                ("wi", ctypes.c_ulonglong), ("sg", ctypes.c_ulonglong), ("footprint", ctypes.c_ulonglong)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_counts.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
                                       ctypes.POINTER(_Orec), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        _lib.oracle_counts.restype = ctypes.c_int
        _lib.oracle_counts_twin.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong),
                                            ctypes.c_int, ctypes.POINTER(_Orec), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]
        _lib.oracle_counts_twin.restype = ctypes.c_int
        _lib.oracle_count_example.argtypes = [ctypes.c_longlong, ctypes.c_longlong]
        _lib.oracle_count_example.restype = ctypes.c_longlong
        assert _lib.oracle_sizeof_orec() == ctypes.sizeof(_Orec)
    return _lib


# Parameter order of each kernel family in enum.c and its static
# work-group / grid dimensionality (used to print stride fields).
KERNELS = {
    "stream": (("dtype", "vec", "N", "s", "L", "shape", "W"), None),
    "fma": (("dtype", "op", "F", "G"), (1, 1)),
    "smem": (("R", "sync", "G"), (1, 1)),
    "barrier": (("B", "G"), (1, 1)),
    "overlap": (("m", "N"), (1, 1)),
    "empty": (("G",), (1, 1)),
}
for _k in ("mm_pf", "mm_nopf", "mm_pf_a", "mm_pf_b", "mm_nopf_a", "mm_nopf_b"):
    KERNELS[_k] = (("n",), (2, 2))
for _k in ("dg_nopf", "dg_dmpf", "dg_nopf_u", "dg_nopf_dm", "dg_dmpf_u", "dg_dmpf_dm", "dg_res",
           "dg_upf", "dg_dmpft", "dg_upf_u", "dg_dmpft_u", "dg_dmpft_res"):
    KERNELS[_k] = (("Np", "Nel", "L0", "L1"), (2, 2))
for _k in ("fd_tile", "fd_direct", "fd_tile_u", "fd_tile_res", "fd_direct_u", "fd_direct_res",
           "fd_tile18", "fd_tile18_u", "fd_tile18_res"):
    KERNELS[_k] = (("n",), (2, 2))

KERNELS["mm_simt"] = (("n", "BM", "BN", "BK"), (2, 2))
KERNELS["mm_tc"] = (("n",), (1, 2))
KERNELS["mm_tc256"] = (("n",), (1, 2))
KERNELS["dg_tile"] = (("Np", "Nel"), (2, 2))
KERNELS["dg_tc"] = (("Np", "Nel", "P", "A"), (1, 2))
KERNELS["fd_block"] = (("n", "BX", "BY", "V"), (2, 2))
KERNELS["smem2d"] = (("R", "T", "G"), (2, 1))

# default parameter values (dtype 0 = float32)
DEFAULTS = {"dtype": 0, "vec": 0, "s": 1, "L": 1, "shape": 0, "W": 16, "op": 2, "sync": 0, "L0": 16, "L1": 16,
            "BX": 64, "BY": 8, "T": 16, "V": 4, "P": 0, "A": -1}


def dims(kernel, params):
    if kernel == "stream":
        return (1, 2) if params.get("shape", 0) == 0 else (2, 2)
    return KERNELS[kernel][1]


def raw_counts(kernel, remove=None, **params):
    """Enumerate the loop domain of `kernel`; returns a list of record dicts.
    remove: global-access tags for work removal (Algorithm 3): the counts are
    then those of the twin derived from `kernel`'s descriptor."""
    names = KERNELS[kernel][0]
    vals = []
    for nm in names:
        v = params.get(nm, DEFAULTS.get(nm))
        if v is None:
            raise ValueError("missing parameter %r for %s" % (nm, kernel))
        vals.append(int(v))
    arr = (ctypes.c_longlong * 8)(*vals)
    cap = 256
    out = (_Orec * cap)()
    n = ctypes.c_int(0)
    if remove is None:
        rc = lib().oracle_counts(kernel.encode(), arr, len(vals), out, cap, ctypes.byref(n))
    else:
        rc = lib().oracle_counts_twin(kernel.encode(), "|".join(remove).encode(), arr, len(vals), out, cap,
                                      ctypes.byref(n))
    if rc != 0:
        raise ValueError("oracle_counts(%s, %r) failed: %d" % (kernel, params, rc))
    recs = []
    for i in range(n.value):
        r = out[i]
        recs.append(dict(kind=r.kind, name=r.name.decode(), dtype=r.dtype.decode(), mem=r.mem, dir=r.dir,
                         dsize=r.dsize, uniform=r.uniform, affine=r.affine, lstr=tuple(r.lstr),
                         gstr=tuple(r.gstr), loopstr=r.loopstr, wi=r.wi, sg=r.sg, footprint=r.footprint))
    return recs


def count_example(n, p):
    """Brute-force count of {(i, j): p <= i < n, p <= j < i + 1}."""
    return lib().oracle_count_example(n, p)
