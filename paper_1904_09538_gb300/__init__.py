"""GB300-native performance modeling (arXiv 1904.09538): Python binding of
libpm.so.  Argument marshalling only -- every step (counts, kernels, timing,
fits, prediction) runs in the C/CUDA library.  PyTorch supplies device memory
and streams.  Names follow include/pm.h without the ``pm_`` prefix."""
import ctypes

import numpy as np

from ._lib import (lib, check, PMError, pm_param, pm_buffer, pm_feature, pm_run_opts, pm_timing, pm_fit_opts,
                   pm_fit_report)

__all__ = ["kernel_lookup", "kernel_names", "counts", "kernel_buffers", "launch", "run", "run_host", "Model",
           "FitPlan", "fit_batched", "counts_desc_interp", "fit_batched_noalloc", "NOALLOC_SCRATCH_BYTES", "PMError", "DTYPES"]

NOALLOC_SCRATCH_BYTES = 8 << 20

DTYPES = {0: np.float32, 1: np.float64, 2: np.uint16}
_KIND = {0: "op", 1: "mem", 2: "sync", 3: "groups", 4: "launch"}
_GRAN = {0: "WI", 1: "SG", 2: "WG", 3: "K"}


def kernel_lookup(name):
    k = ctypes.c_int32()
    check(lib().pm_kernel_lookup(name.encode(), ctypes.byref(k)))
    return k.value


def kernel_names():
    n = ctypes.c_int32()
    check(lib().pm_kernel_count(ctypes.byref(n)))
    out = []
    for i in range(n.value):
        s = ctypes.c_char_p()
        check(lib().pm_kernel_name(i, ctypes.byref(s)))
        out.append(s.value.decode())
    return out


def _params(params):
    keys = [k.encode() for k in params]
    arr = (pm_param * max(1, len(params)))()
    for i, (k, v) in enumerate(params.items()):
        arr[i].key = keys[i]
        arr[i].value = float(v)
    return arr, len(params), keys


def _kid(kernel):
    return kernel if isinstance(kernel, int) else kernel_lookup(kernel)


def _records(out, count):
    recs = []
    for i in range(count):
        f = out[i]
        r = dict(name=f.name.decode(), kind=_KIND[f.kind], gran=_GRAN[f.gran], count=f.count)
        if f.kind == 0:
            r.update(dtype=f.dtype.decode(), op=f.op.decode(), count_wi=f.count_wi, count_sg=f.count_sg)
        elif f.kind == 1:
            r.update(tag=f.tag.decode(), mem="local" if f.mem else "global", dtype=f.dtype.decode(),
                     dir="store" if f.dir else "load", dsize=f.dsize, lstr=tuple(f.lstride[:f.nl]),
                     gstr=tuple(f.gstride[:f.ng]), loopstr=f.loop_stride, accesses=f.accesses,
                     footprint=f.footprint, count_wi=f.count_wi, count_sg=f.count_sg)
        recs.append(r)
    return recs


def counts(kernel, **params):
    """Exact feature records (pm_counts) as dicts."""
    out, n = _counts_raw(kernel, **params)
    return _records(out, n)


def _counts_desc_raw(description, interp=None, **params):
    arr, n, _keep = _params(params)
    interp = interp or {}
    names = [k.encode() for k in interp]
    ip = (_lib.pm_interp * max(1, len(interp)))()
    for i, (k, pd) in enumerate(interp.items()):
        period, degree = (None, None) if pd is None else pd
        ip[i] = _lib.pm_interp(names[i], 0 if period is None else int(period), -1 if degree is None else int(degree))
    cap = 64
    while True:
        out = (pm_feature * cap)()
        nout = ctypes.c_size_t()
        st = lib().pm_counts_desc(description.encode(), arr, n, ip, len(interp), out, cap, ctypes.byref(nout))
        if st == -9 and nout.value > cap:
            cap = nout.value
            continue
        check(st)
        return out, nout.value


def counts_desc(description, interp=None, **params):
    """Exact feature records of a kernel given as a loop-nest description
    (pm_counts_desc).  interp: {parameter: (period, degree bound)} for sizes
    too large to enumerate; None (or None in either place) lets the library
    derive it from the description."""
    return _records(*_counts_desc_raw(description, interp, **params))


def counts_desc_interp(description, param, **params):
    """(period, degree bound) of the counts in `param`, derived from the
    description (pm_counts_desc_interp)."""
    arr, n, _keep = _params(params)
    pe, de = ctypes.c_int32(), ctypes.c_int32()
    check(lib().pm_counts_desc_interp(description.encode(), param.encode(), arr, n, ctypes.byref(pe),
                                      ctypes.byref(de)))
    return pe.value, de.value


def _counts_raw(kernel, **params):
    arr, n, _keep = _params(params)
    cap = 64
    out = (pm_feature * cap)()
    nout = ctypes.c_size_t()
    check(lib().pm_counts(_kid(kernel), arr, n, out, cap, ctypes.byref(nout)))
    return out, nout.value


def kernel_buffers(kernel, **params):
    arr, n, _keep = _params(params)
    cap = 16
    out = (pm_buffer * cap)()
    nout = ctypes.c_size_t()
    check(lib().pm_kernel_buffers(_kid(kernel), arr, n, out, cap, ctypes.byref(nout)))
    return [dict(name=out[i].name.decode(), dtype=DTYPES[out[i].dtype], role="in" if out[i].role == 0 else "out",
                 elems=out[i].elems) for i in range(nout.value)]


def _ptrs(bufs):
    ptrs = (ctypes.c_void_p * max(1, len(bufs)))()
    for i, b in enumerate(bufs):
        if hasattr(b, "data_ptr"):
            if not b.is_cuda or not b.is_contiguous():
                raise ValueError("buffer %d must be a contiguous CUDA tensor" % i)
            ptrs[i] = b.data_ptr()
        else:
            ptrs[i] = int(b)
    return ptrs


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(stream)


def resources(kernel, **params):
    """Compiled resources and launch shape of a kernel instance
    (pm_kernel_resources; needs a CUDA device, launches nothing)."""
    arr, n, _keep = _params(params)
    r = _lib.pm_resources()
    check(lib().pm_kernel_resources(_kid(kernel), arr, n, ctypes.byref(r)))
    return {f: int(getattr(r, f)) for f, _ in r._fields_}


def launch(kernel, bufs, stream=None, **params):
    """Enqueue one launch (device buffers in pm_kernel_buffers order)."""
    arr, n, _keep = _params(params)
    check(lib().pm_launch(_kid(kernel), arr, n, _ptrs(bufs), len(bufs), _stream(stream)))


def run(kernel, bufs, warmup=2, trials=60, outlier_factor=5.0, stream=None, want_trials=False, flush_l2=False,
        **params):
    """Device-timed trials (pm_run).  Returns a timing dict (ms)."""
    arr, n, _keep = _params(params)
    opts = pm_run_opts(warmup, trials, outlier_factor, 1 if flush_l2 else 0)
    tm = pm_timing()
    tr = (ctypes.c_float * trials)()
    check(lib().pm_run(_kid(kernel), arr, n, _ptrs(bufs), len(bufs), ctypes.byref(opts), _stream(stream), tr,
                       ctypes.byref(tm)))
    out = dict(mean_ms=tm.mean_ms, median_ms=tm.median_ms, min_ms=tm.min_ms, max_ms=tm.max_ms,
               n_trials=tm.n_trials, n_dropped=tm.n_dropped)
    if want_trials:
        out["trials_ms"] = list(tr)
    return out


def probe_latency(buf, hops=100000, stream=None):
    """pm_probe_latency on a device tensor (its bytes are overwritten): mean
    nanoseconds per dependent load from the level that holds it."""
    ns = ctypes.c_double()
    check(lib().pm_probe_latency(ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(), int(hops),
                                 ctypes.byref(ns), _stream(stream)))
    return ns.value


def run_host(kernel, host_arrays, warmup=2, trials=60, outlier_factor=5.0, stream=None, flush_l2=False, **params):
    """pm_run with host (NumPy) buffers: copies in, runs, copies out."""
    arr, n, _keep = _params(params)
    ptrs = (ctypes.c_void_p * max(1, len(host_arrays)))()
    for i, a in enumerate(host_arrays):
        if hasattr(a, "data_ptr"):
            ptrs[i] = a.data_ptr()
        else:
            if not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host array %d must be C-contiguous" % i)
            ptrs[i] = a.ctypes.data
    opts = pm_run_opts(warmup, trials, outlier_factor, 1 if flush_l2 else 0)
    tm = pm_timing()
    cms = ctypes.c_double()
    check(lib().pm_run_host(_kid(kernel), arr, n, ptrs, len(host_arrays), ctypes.byref(opts), _stream(stream),
                            None, ctypes.byref(tm), ctypes.byref(cms)))
    return dict(mean_ms=tm.mean_ms, median_ms=tm.median_ms, min_ms=tm.min_ms, n_trials=tm.n_trials,
                n_dropped=tm.n_dropped, copy_ms=cms.value)


def _host_jobs(jobs):
    keep = []
    arr = (_lib.pm_host_job * max(1, len(jobs)))()
    for i, (kernel, host_arrays, params) in enumerate(jobs):
        parr, n, k = _params(params)
        ptrs = (ctypes.c_void_p * max(1, len(host_arrays)))()
        for b, a in enumerate(host_arrays):
            if a is None:                      # an output left on the device
                ptrs[b] = None
            elif hasattr(a, "data_ptr"):
                ptrs[b] = a.data_ptr()
            else:
                if not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("job %d host array %d must be C-contiguous" % (i, b))
                ptrs[b] = a.ctypes.data
        keep += [parr, k, ptrs]
        arr[i] = _lib.pm_host_job(_kid(kernel), ctypes.cast(parr, ctypes.c_void_p), n,
                                  ctypes.cast(ptrs, ctypes.c_void_p), len(host_arrays))
    return arr, keep


def run_host_batch(jobs, warmup=0, trials=1, outlier_factor=5.0, stream=None, flush_l2=False):
    """pm_run_host over a list of (kernel, host_arrays, params) jobs with the
    output copy of each job overlapping the input copy of the next; None for
    an output array leaves that output on the device; an input region that
    several jobs read from the same host address is copied once.  Returns
    (list of timing dicts, copy_ms)."""
    arr, keep = _host_jobs(jobs)
    opts = pm_run_opts(warmup, trials, outlier_factor, 1 if flush_l2 else 0)
    tms = (pm_timing * max(1, len(jobs)))()
    cms = ctypes.c_double()
    check(lib().pm_run_host_batch(arr, len(jobs), ctypes.byref(opts), _stream(stream), tms, ctypes.byref(cms)))
    return [dict(mean_ms=t.mean_ms, median_ms=t.median_ms, min_ms=t.min_ms, n_trials=t.n_trials,
                 n_dropped=t.n_dropped) for t in tms[:len(jobs)]], cms.value


def run_host_batch_bytes(jobs):
    """(host->device, device->host) bytes run_host_batch copies for these
    jobs (shared input regions counted once).  Host only."""
    arr, keep = _host_jobs(jobs)
    h2d, d2h = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().pm_run_host_batch_bytes(arr, len(jobs), ctypes.byref(h2d), ctypes.byref(d2h)))
    return int(h2d.value), int(d2h.value)


def _opts(max_iter=200, ftol=1e-15, xtol=1e-12, p0=None):
    return pm_fit_opts(max_iter, ftol, xtol, 0 if p0 is None else 1)


def _report(r):
    return dict(status=r.status, iterations=r.iterations, rank=r.rank, linear=bool(r.linear), residual=r.residual,
                lambda_=r.lambda_, cond=r.cond)


class Model:
    """Output feature + expression over f_* features and p_* parameters."""

    def __init__(self, out_feature, expr):
        h = ctypes.c_void_p()
        check(lib().pm_model_create(out_feature.encode(), expr.encode(), ctypes.byref(h)))
        self._h = h
        self.out_feature, self.expr = out_feature, expr
        nf, np_ = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib().pm_model_info(h, ctypes.byref(nf), ctypes.byref(np_)))
        self.features, self.params = [], []
        s = ctypes.c_char_p()
        for i in range(nf.value):
            check(lib().pm_model_feature_name(h, i, ctypes.byref(s)))
            self.features.append(s.value.decode())
        for i in range(np_.value):
            check(lib().pm_model_param_name(h, i, ctypes.byref(s)))
            self.params.append(s.value.decode())
        li = ctypes.c_int32()
        check(lib().pm_model_is_linear(h, ctypes.byref(li)))
        self.is_linear = bool(li.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().pm_model_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def feature_values_desc(self, description, interp=None, **params):
        """One design-matrix row on a kernel given as a loop-nest description."""
        feats, n = _counts_desc_raw(description, interp, **params)
        row = (ctypes.c_double * max(1, len(self.features)))()
        check(lib().pm_feature_values(self._h, feats, n, row))
        return np.array(row[:len(self.features)], dtype=np.float64)

    def feature_values(self, kernel, **params):
        """One design-matrix row: this model's features on kernel(params)."""
        feats, n = _counts_raw(kernel, **params)
        row = (ctypes.c_double * max(1, len(self.features)))()
        check(lib().pm_feature_values(self._h, feats, n, row))
        return np.array(row[:len(self.features)], dtype=np.float64)

    def fit(self, X, t, p0=None, max_iter=200, ftol=1e-15, xtol=1e-12, raise_on_status=False):
        """pm_fit on host arrays.  Returns (p, report)."""
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(len(t), len(self.features))
        t = np.ascontiguousarray(t, dtype=np.float64)
        p = np.zeros(len(self.params)) if p0 is None else np.array(p0, dtype=np.float64)
        rep = pm_fit_report()
        opts = _opts(max_iter, ftol, xtol, p0)
        st = lib().pm_fit(self._h, X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t), ctypes.byref(opts),
                          p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(rep))
        if st != 0 and (raise_on_status or st not in (-4, -5)):
            check(st)
        return p, _report(rep)

    def predict(self, p, X):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, len(self.features))
        p = np.ascontiguousarray(p, dtype=np.float64)
        out = np.empty(X.shape[0])
        check(lib().pm_predict(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), X.shape[0],
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out


class FitPlan:
    """Batched calibration plan: one persistent launch, replayed from a CUDA graph."""

    def __init__(self, models, rows, p0_given=False, threads=0, max_iter=200, ftol=1e-15, xtol=1e-12):
        self.models = list(models)
        self.rows = [int(r) for r in rows]
        hs = (ctypes.c_void_p * len(self.models))(*[m.handle.value for m in self.models])
        rw = (ctypes.c_size_t * len(self.rows))(*self.rows)
        opts = pm_fit_opts(max_iter, ftol, xtol, 1 if p0_given else 0)
        h = ctypes.c_void_p()
        check(lib().pm_fit_plan_create(hs, len(self.models), rw, ctypes.byref(opts), threads, ctypes.byref(h)))
        self._h = h
        self.nparams = [len(m.params) for m in self.models]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().pm_fit_plan_destroy(h)
            self._h = None

    def run(self, X_concat, t_concat, p_concat=None, stream=None):
        X = np.ascontiguousarray(X_concat, dtype=np.float64)
        t = np.ascontiguousarray(t_concat, dtype=np.float64)
        p = np.zeros(sum(self.nparams)) if p_concat is None else np.array(p_concat, dtype=np.float64)
        reps = (pm_fit_report * len(self.models))()
        D = ctypes.POINTER(ctypes.c_double)
        check(lib().pm_fit_plan_run(self._h, X.ctypes.data_as(D), t.ctypes.data_as(D), p.ctypes.data_as(D), reps,
                                    _stream(stream) if stream is not None else ctypes.c_void_p(0)))
        return p, [_report(r) for r in reps]


def fit_batched(models, Xs, ts, p0s=None, threads=0, **kw):
    """Fit models[k] on (Xs[k], ts[k]) in one batched launch."""
    plan = FitPlan(models, [len(t) for t in ts], p0_given=p0s is not None, threads=threads, **kw)
    X = np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in Xs]) if Xs else np.zeros(0)
    t = np.concatenate([np.asarray(x, dtype=np.float64) for x in ts])
    p0 = None if p0s is None else np.concatenate([np.asarray(p, dtype=np.float64) for p in p0s])
    p, reps = plan.run(X, t, p0)
    out, o = [], 0
    for n in plan.nparams:
        out.append(p[o:o + n])
        o += n
    return out, reps


def fit_batched_noalloc(models, Xs, ts, p0s=None, max_iter=200, ftol=1e-15, xtol=1e-12, stream=None):
    """pm_fit_batched_noalloc: the batched fit staged in the library's static
    device scratch (no GPU memory allocation; see include/pm.h for who needs
    it and its limits).  Same arguments and results as fit_batched."""
    models = list(models)
    rows = [len(t) for t in ts]
    X = np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in Xs]) if Xs else np.zeros(0)
    t = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in ts]))
    nps = [len(m.params) for m in models]
    p = np.zeros(sum(nps)) if p0s is None else np.ascontiguousarray(
        np.concatenate([np.asarray(q, dtype=np.float64) for q in p0s]))
    X = np.ascontiguousarray(X)
    hs = (ctypes.c_void_p * len(models))(*[m.handle.value for m in models])
    rw = (ctypes.c_size_t * len(rows))(*rows)
    opts = pm_fit_opts(max_iter, ftol, xtol, 0 if p0s is None else 1)
    reps = (pm_fit_report * len(models))()
    D = ctypes.POINTER(ctypes.c_double)
    check(lib().pm_fit_batched_noalloc(hs, len(models), X.ctypes.data_as(D), t.ctypes.data_as(D), rw,
                                       ctypes.byref(opts), p.ctypes.data_as(D), reps,
                                       _stream(stream) if stream is not None else ctypes.c_void_p(0)))
    out, o = [], 0
    for n in nps:
        out.append(p[o:o + n])
        o += n
    return out, [_report(r) for r in reps]
