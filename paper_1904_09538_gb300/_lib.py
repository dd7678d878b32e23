"""ctypes declarations of libpm.so (include/pm.h).  Loading fails loudly if
the in-tree library has not been built; there is no fallback."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_build", "libpm.so")

c_size_t = ctypes.c_size_t


class pm_param(ctypes.Structure):
    _fields_ = [("key", ctypes.c_char_p), ("value", ctypes.c_double)]


class pm_buffer(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("dtype", ctypes.c_int32), ("role", ctypes.c_int32),
                ("elems", ctypes.c_uint64)]


class pm_feature(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 192), ("kind", ctypes.c_int32), ("gran", ctypes.c_int32),
                ("count", ctypes.c_uint64), ("count_wi", ctypes.c_uint64), ("count_sg", ctypes.c_uint64),
                ("tag", ctypes.c_char * 32), ("dtype", ctypes.c_char * 16), ("op", ctypes.c_char * 8),
                ("mem", ctypes.c_int32), ("dir", ctypes.c_int32), ("dsize", ctypes.c_int32),
                ("nl", ctypes.c_int32), ("ng", ctypes.c_int32),
                ("lstride", ctypes.c_int64 * 3), ("gstride", ctypes.c_int64 * 3), ("loop_stride", ctypes.c_int64),
                ("accesses", ctypes.c_uint64), ("footprint", ctypes.c_uint64)]


class pm_resources(ctypes.Structure):
    _fields_ = [("regs_per_thread", ctypes.c_int32), ("local_bytes_per_thread", ctypes.c_int32),
                ("static_smem_bytes", ctypes.c_int32), ("dynamic_smem_bytes", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("max_threads_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("sm_count", ctypes.c_int32), ("grid_blocks", ctypes.c_uint64)]


class pm_interp(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("period", ctypes.c_int32), ("degree", ctypes.c_int32)]


class pm_host_job(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("p", ctypes.c_void_p), ("np", ctypes.c_size_t),
                ("host_bufs", ctypes.c_void_p), ("nbufs", ctypes.c_size_t)]


class pm_run_opts(ctypes.Structure):
    _fields_ = [("warmup", ctypes.c_int32), ("trials", ctypes.c_int32), ("outlier_factor", ctypes.c_double),
                ("flush_l2", ctypes.c_int32)]


class pm_timing(ctypes.Structure):
    _fields_ = [("mean_ms", ctypes.c_double), ("median_ms", ctypes.c_double), ("min_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("n_trials", ctypes.c_int32), ("n_dropped", ctypes.c_int32)]


class pm_fit_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("ftol", ctypes.c_double), ("xtol", ctypes.c_double),
                ("use_p0", ctypes.c_int32)]


class pm_fit_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("linear", ctypes.c_int32), ("residual", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("cond", ctypes.c_double)]


P = ctypes.POINTER
vp = ctypes.c_void_p
i32 = ctypes.c_int32
dp = P(ctypes.c_double)
fp = P(ctypes.c_float)

# name -> (restype, argtypes)
SIGNATURES = {
    "pm_last_error": (ctypes.c_char_p, []),
    "pm_test_fail_allocation": (i32, [i32]),
    "pm_test_bounded_wait": (i32, [ctypes.c_int64, vp]),
    "pm_kernel_lookup": (i32, [ctypes.c_char_p, P(i32)]),
    "pm_kernel_count": (i32, [P(i32)]),
    "pm_kernel_name": (i32, [i32, P(ctypes.c_char_p)]),
    "pm_kernel_buffers": (i32, [i32, P(pm_param), c_size_t, P(pm_buffer), c_size_t, P(c_size_t)]),
    "pm_counts": (i32, [i32, P(pm_param), c_size_t, P(pm_feature), c_size_t, P(c_size_t)]),
    "pm_counts_desc": (i32, [ctypes.c_char_p, P(pm_param), c_size_t, P(pm_interp), c_size_t, P(pm_feature), c_size_t,
                             P(c_size_t)]),
    "pm_counts_desc_interp": (i32, [ctypes.c_char_p, ctypes.c_char_p, P(pm_param), c_size_t, P(i32), P(i32)]),
    "pm_launch": (i32, [i32, P(pm_param), c_size_t, P(vp), c_size_t, vp]),
    "pm_kernel_resources": (i32, [i32, P(pm_param), c_size_t, P(pm_resources)]),
    "pm_run": (i32, [i32, P(pm_param), c_size_t, P(vp), c_size_t, P(pm_run_opts), vp, fp, P(pm_timing)]),
    "pm_run_host": (i32, [i32, P(pm_param), c_size_t, P(vp), c_size_t, P(pm_run_opts), vp, fp, P(pm_timing), dp]),
    "pm_run_host_batch": (i32, [P(pm_host_job), c_size_t, P(pm_run_opts), vp, P(pm_timing), dp]),
    "pm_run_host_batch_bytes": (i32, [P(pm_host_job), c_size_t, P(ctypes.c_uint64), P(ctypes.c_uint64)]),
    "pm_probe_latency": (i32, [vp, c_size_t, i32, dp, vp]),
    "pm_model_create": (i32, [ctypes.c_char_p, ctypes.c_char_p, P(vp)]),
    "pm_model_destroy": (None, [vp]),
    "pm_model_info": (i32, [vp, P(c_size_t), P(c_size_t)]),
    "pm_model_feature_name": (i32, [vp, c_size_t, P(ctypes.c_char_p)]),
    "pm_model_param_name": (i32, [vp, c_size_t, P(ctypes.c_char_p)]),
    "pm_model_is_linear": (i32, [vp, P(i32)]),
    "pm_feature_values": (i32, [vp, P(pm_feature), c_size_t, dp]),
    "pm_fit": (i32, [vp, dp, dp, c_size_t, P(pm_fit_opts), dp, P(pm_fit_report)]),
    "pm_fit_plan_create": (i32, [P(vp), c_size_t, P(c_size_t), P(pm_fit_opts), i32, P(vp)]),
    "pm_fit_plan_run": (i32, [vp, dp, dp, dp, P(pm_fit_report), vp]),
    "pm_fit_plan_destroy": (None, [vp]),
    "pm_fit_batched": (i32, [P(vp), c_size_t, dp, dp, P(c_size_t), P(pm_fit_opts), dp, P(pm_fit_report), vp]),
    "pm_fit_batched_noalloc": (i32, [P(vp), c_size_t, dp, dp, P(c_size_t), P(pm_fit_opts), dp, P(pm_fit_report), vp]),
    "pm_residual": (i32, [vp, vp, vp, c_size_t, vp, vp, vp]),
    "pm_residual_vjp": (i32, [vp, vp, vp, c_size_t, vp, vp, vp, vp]),
    "pm_jacobian": (i32, [vp, vp, vp, c_size_t, vp, vp, vp]),
    "pm_lm_init": (i32, [vp, dp, P(pm_fit_opts), vp, vp, vp]),
    "pm_lm_step": (i32, [vp, vp, vp, vp, c_size_t, vp, vp]),
    "pm_lm_update": (i32, [vp, vp, c_size_t, vp, vp, vp]),
    "pm_lm_report": (i32, [vp, P(pm_fit_report), vp]),
    "pm_predict": (i32, [vp, dp, dp, c_size_t, dp]),
}

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(SO):
            raise ImportError("libpm.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"`"
                              % SO)
        L = ctypes.CDLL(SO)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


STATUS = {0: "PM_OK", -1: "PM_EINVAL", -2: "PM_ENOMEM", -3: "PM_ECUDA", -4: "PM_ENOTCONV", -5: "PM_ERANK",
          -6: "PM_ETIMEOUT", -7: "PM_EUNKNOWN_KERNEL", -8: "PM_EPARSE", -9: "PM_ECAP"}


class PMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def check(status):
    if status != 0:
        raise PMError(status, lib().pm_last_error().decode(errors="replace"))
    return status
