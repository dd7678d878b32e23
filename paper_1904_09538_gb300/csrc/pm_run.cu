// pm_launch / pm_run / pm_run_host: stream-ordered launches and the paper's
// wall-time feature (Section "Other Features": 60 trials averaged, excluding
// host-device transfer; Section "Results": anomalous ~10x trials excluded).
#include <algorithm>
#include <cmath>
#include <cuda_runtime.h>
#include <mutex>
#include <string>
#include <vector>

#include "pm_internal.h"

namespace pm {

static pm_status launch_any(const KP &kp, void *const *bufs, size_t nbufs, void *stream) {
    pm_status s = validate(kp);
    if (s) return s;
    std::vector<BufSpec> spec;
    if ((s = buffers(kp, spec))) return s;
    if (nbufs != spec.size())
        return fail(PM_EINVAL, "%s: %zu buffers passed, %zu needed", kp.def->name, nbufs, spec.size());
    for (size_t i = 0; i < spec.size(); i++)
        if (!bufs[i]) return fail(PM_EINVAL, "%s: buffer %zu (%s) is NULL", kp.def->name, i, spec[i].name);
    switch (kp.def->fam) {
    case FAM_MM: case FAM_DG: case FAM_FD: return launch_modeled(kp, bufs, stream);
    case FAM_SIMT: case FAM_FDB: case FAM_DGT: return launch_tiles(kp, bufs, stream);
    case FAM_TC: return launch_tc(kp, bufs, stream);
    case FAM_DGC: return launch_dgc(kp, bufs, stream);
    default: return launch_suite(kp, bufs, stream);
    }
}

static size_t dtype_size(int dt) { return dt == PM_F32 ? 4 : dt == PM_F64 ? 8 : 2; }

// pm_run_host stages through the device's default memory pool; keeping the
// freed staging memory reserved (instead of unmapping it at every
// synchronisation) saves remapping gigabytes on every call.
pm_status retain_staging_pool() {
    static bool done[64];
    static std::mutex mu;
    int dev = 0;
    PM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return PM_OK;
    cudaMemPool_t pool;
    PM_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t keep = UINT64_MAX;
    PM_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    done[dev] = true;
    return PM_OK;
}

thread_local LaunchQuery *g_launch_query = nullptr;

bool launch_query_hook(const void *fn, unsigned gx, unsigned gy, unsigned gz, unsigned bx, unsigned by, unsigned bz,
                       size_t smem) {
    LaunchQuery *q = g_launch_query;
    if (!q) return false;
    q->hits++;
    cudaFuncAttributes a;
    int dev = 0, sms = 0, nb = 0;
    const int threads = (int)(bx * by * bz);
    if (cudaFuncGetAttributes(&a, fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        q->status = fail(PM_ECUDA, "pm_kernel_resources: attribute query failed");
        return true;
    }
    pm_resources *o = q->out;
    o->regs_per_thread = a.numRegs;
    o->local_bytes_per_thread = (int32_t)a.localSizeBytes;
    o->static_smem_bytes = (int32_t)a.sharedSizeBytes;
    o->dynamic_smem_bytes = (int32_t)smem;
    o->threads_per_block = threads;
    o->max_threads_per_block = a.maxThreadsPerBlock;
    o->blocks_per_sm = nb;
    o->sm_count = sms;
    o->grid_blocks = (uint64_t)gx * gy * gz;
    return true;
}

// L2 flush: overwrite a buffer larger than the 129 MB L2 (one per device).
constexpr size_t kFlushBytes = 256u << 20;
static void *g_flush[64];
static std::mutex g_flush_mu;

__global__ void k_l2_flush(int4 *__restrict__ p, size_t n, int v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = make_int4(v, v, v, v);
}

static pm_status flush_l2(cudaStream_t st) {
    int dev = 0;
    PM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PM_EINVAL, "flush_l2: device ordinal %d unsupported", dev);
    void *buf = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_flush_mu);
        if (!g_flush[dev]) {
            if (alloc_fault_injected() || cudaMalloc(&g_flush[dev], kFlushBytes) != cudaSuccess) {
                g_flush[dev] = nullptr;
                return fail(PM_ENOMEM, "flush_l2: cannot allocate the %zu-byte flush buffer", kFlushBytes);
            }
        }
        buf = g_flush[dev];
    }
    static int counter = 0;
    k_l2_flush<<<4 * 152, 512, 0, st>>>((int4 *)buf, kFlushBytes / sizeof(int4), ++counter);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

struct EventPool {
    std::vector<cudaEvent_t> ev;
    ~EventPool() {
        for (auto e : ev) cudaEventDestroy(e);
    }
    pm_status make(size_t n) {
        ev.resize(n, nullptr);
        for (size_t i = 0; i < n; i++) PM_CUDA_TRY(cudaEventCreate(&ev[i]));
        return PM_OK;
    }
};

static pm_status timed(const KP &kp, void *const *bufs, size_t nbufs, const pm_run_opts *opts, void *stream,
                       float *trial_ms, pm_timing *out) {
    pm_run_opts o{2, 60, 5.0, 0};
    if (opts) o = *opts;
    if (o.warmup < 0 || o.trials < 1 || o.trials > 100000)
        return fail(PM_EINVAL, "pm_run: need warmup >= 0 and 1 <= trials <= 100000");
    cudaStream_t st = (cudaStream_t)stream;
    pm_status s;
    for (int w = 0; w < o.warmup; w++)
        if ((s = launch_any(kp, bufs, nbufs, stream))) return s;
    EventPool pool;
    if ((s = pool.make(2 * (size_t)o.trials))) return s;
    for (int t = 0; t < o.trials; t++) {
        if (o.flush_l2 && (s = flush_l2(st))) return s;
        PM_CUDA_TRY(cudaEventRecord(pool.ev[2 * t], st));
        if ((s = launch_any(kp, bufs, nbufs, stream))) return s;
        PM_CUDA_TRY(cudaEventRecord(pool.ev[2 * t + 1], st));
    }
    PM_CUDA_TRY(cudaEventSynchronize(pool.ev[2 * o.trials - 1]));
    PM_CUDA_TRY(cudaGetLastError());
    if (kp.def->fam == FAM_TC && (s = tc_check_timeout())) return s;
    if (kp.def->fam == FAM_FDB && (s = fdb_check_timeout())) return s;
    if (kp.def->fam == FAM_DGT && (s = dgt_check_timeout())) return s;
    if (kp.def->fam == FAM_DGC && (s = dgc_check_timeout())) return s;
    std::vector<float> ms(o.trials);
    for (int t = 0; t < o.trials; t++) PM_CUDA_TRY(cudaEventElapsedTime(&ms[t], pool.ev[2 * t], pool.ev[2 * t + 1]));
    if (trial_ms)
        for (int t = 0; t < o.trials; t++) trial_ms[t] = ms[t];
    std::vector<float> sorted = ms;
    std::sort(sorted.begin(), sorted.end());
    const double med = o.trials % 2 ? (double)sorted[o.trials / 2]
                                    : 0.5 * ((double)sorted[o.trials / 2 - 1] + (double)sorted[o.trials / 2]);
    double sum = 0.0, mn = 1e300, mx = 0.0;
    int kept = 0;
    for (float v : ms) {
        if (o.outlier_factor > 0 && v > o.outlier_factor * med) continue;
        sum += v;
        mn = std::min(mn, (double)v);
        mx = std::max(mx, (double)v);
        kept++;
    }
    if (out) {
        out->mean_ms = sum / kept;
        out->median_ms = med;
        out->min_ms = mn;
        out->max_ms = mx;
        out->n_trials = o.trials;
        out->n_dropped = o.trials - kept;
    }
    return PM_OK;
}

}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_kernel_resources(int32_t kernel, const pm_param *p, size_t np, pm_resources *out) {
    KP kp;
    pm_status s = parse_params(kernel, p, np, &kp);
    if (s) return s;
    if (!out) return fail(PM_EINVAL, "pm_kernel_resources: out is NULL");
    if ((s = validate(kp))) return s;
    std::vector<BufSpec> spec;
    if ((s = buffers(kp, spec))) return s;
    // placeholder addresses: aligned, never dereferenced (the launch is skipped)
    std::vector<void *> fake(spec.size());
    for (size_t i = 0; i < fake.size(); i++) fake[i] = (void *)(uintptr_t)((i + 1) << 20);
    *out = pm_resources{};
    LaunchQuery q{out, 0, PM_OK};
    g_launch_query = &q;
    s = launch_any(kp, fake.data(), fake.size(), nullptr);
    g_launch_query = nullptr;
    if (s) return s;
    if (q.status) return q.status;
    if (q.hits != 1) return fail(PM_EINVAL, "pm_kernel_resources: %s issued %d launches", kp.def->name, q.hits);
    return PM_OK;
}

pm_status pm_launch(int32_t kernel, const pm_param *p, size_t np, void *const *bufs, size_t nbufs, void *stream) {
    KP kp;
    pm_status s = parse_params(kernel, p, np, &kp);
    if (s) return s;
    if (nbufs && !bufs) return fail(PM_EINVAL, "pm_launch: bufs is NULL");
    return launch_any(kp, bufs, nbufs, stream);
}

pm_status pm_run(int32_t kernel, const pm_param *p, size_t np, void *const *bufs, size_t nbufs,
                 const pm_run_opts *opts, void *stream, float *trial_ms, pm_timing *out) {
    KP kp;
    pm_status s = parse_params(kernel, p, np, &kp);
    if (s) return s;
    if (nbufs && !bufs) return fail(PM_EINVAL, "pm_run: bufs is NULL");
    return timed(kp, bufs, nbufs, opts, stream, trial_ms, out);
}

pm_status pm_run_host(int32_t kernel, const pm_param *p, size_t np, void *const *host_bufs, size_t nbufs,
                      const pm_run_opts *opts, void *stream, float *trial_ms, pm_timing *out, double *copy_ms) {
    KP kp;
    pm_status s = parse_params(kernel, p, np, &kp);
    if (s) return s;
    if ((s = validate(kp))) return s;
    std::vector<BufSpec> spec;
    if ((s = buffers(kp, spec))) return s;
    if (nbufs != spec.size()) return fail(PM_EINVAL, "pm_run_host: %zu buffers passed, %zu needed", nbufs, spec.size());
    for (size_t i = 0; i < nbufs; i++)
        if (!host_bufs[i]) return fail(PM_EINVAL, "pm_run_host: host buffer %zu is NULL", i);
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = retain_staging_pool())) return s;
    std::vector<void *> dev(nbufs, nullptr);
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    pm_status rc = PM_OK;
    float c_in = 0, c_out = 0;
    for (int i = 0; i < 4 && rc == PM_OK; i++)
        if (cudaEventCreate(&e[i]) != cudaSuccess) rc = fail(PM_ECUDA, "pm_run_host: cudaEventCreate failed");
    for (size_t i = 0; i < nbufs && rc == PM_OK; i++)
        if (alloc_fault_injected() || cudaMallocAsync(&dev[i], spec[i].elems * dtype_size(spec[i].dtype), st) != cudaSuccess)
            rc = fail(PM_ENOMEM, "pm_run_host: cudaMallocAsync of %s failed", spec[i].name);
    if (rc == PM_OK) cudaEventRecord(e[0], st);
    for (size_t i = 0; i < nbufs && rc == PM_OK; i++)
        if (spec[i].role == PM_IN &&
            cudaMemcpyAsync(dev[i], host_bufs[i], spec[i].elems * dtype_size(spec[i].dtype), cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
            rc = fail(PM_ECUDA, "pm_run_host: host-to-device copy of %s failed", spec[i].name);
    if (rc == PM_OK) cudaEventRecord(e[1], st);
    if (rc == PM_OK) rc = timed(kp, dev.data(), nbufs, opts, stream, trial_ms, out);
    if (rc == PM_OK) cudaEventRecord(e[2], st);
    for (size_t i = 0; i < nbufs && rc == PM_OK; i++)
        if (spec[i].role == PM_OUT &&
            cudaMemcpyAsync(host_bufs[i], dev[i], spec[i].elems * dtype_size(spec[i].dtype), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess)
            rc = fail(PM_ECUDA, "pm_run_host: device-to-host copy of %s failed", spec[i].name);
    if (rc == PM_OK) {
        cudaEventRecord(e[3], st);
        if (cudaEventSynchronize(e[3]) != cudaSuccess) rc = fail(PM_ECUDA, "pm_run_host: synchronize failed");
    }
    if (rc == PM_OK) {
        cudaEventElapsedTime(&c_in, e[0], e[1]);
        cudaEventElapsedTime(&c_out, e[2], e[3]);
        if (copy_ms) *copy_ms = (double)c_in + (double)c_out;
    }
    for (size_t i = 0; i < nbufs; i++)
        if (dev[i]) cudaFreeAsync(dev[i], st);
    cudaStreamSynchronize(st);
    for (int i = 0; i < 4; i++)
        if (e[i]) cudaEventDestroy(e[i]);
    return rc;
}

}  // extern "C"

namespace {

struct BatchJob {
    KP kp;
    std::vector<BufSpec> spec;
    std::vector<int> shared;   // per buffer: index into the shared inputs, or -1
};

// An input region several jobs of a batch read: every input buffer that
// starts at the same host address.  It is copied once, at the largest extent
// any of its readers reads; all regions are copied back to back at the start
// of the batch.
struct SharedIn {
    const char *host;
    size_t bytes;
    int readers;
    void *dev;
};

size_t buf_bytes(const BufSpec &b) { return b.elems * dtype_size(b.dtype); }

pm_status batch_plan(const char *who, const pm_host_job *jobs, size_t njobs, std::vector<BatchJob> &J,
                     std::vector<SharedIn> &sh) {
    if (njobs && !jobs) return fail(PM_EINVAL, "%s: jobs is NULL", who);
    J.assign(njobs, BatchJob{});
    pm_status s;
    for (size_t i = 0; i < njobs; i++) {
        const pm_host_job &h = jobs[i];
        if ((s = parse_params(h.kernel, h.p, h.np, &J[i].kp))) return s;
        if ((s = validate(J[i].kp))) return s;
        if ((s = buffers(J[i].kp, J[i].spec))) return s;
        if (h.nbufs != J[i].spec.size())
            return fail(PM_EINVAL, "%s: job %zu: %zu buffers passed, %zu needed", who, i, h.nbufs, J[i].spec.size());
        for (size_t b = 0; b < h.nbufs; b++)
            if (!h.host_bufs || (!h.host_bufs[b] && J[i].spec[b].role == PM_IN))
                return fail(PM_EINVAL, "%s: job %zu input buffer %zu is NULL", who, i, b);
    }
    // group the inputs by host start address
    sh.clear();
    for (size_t i = 0; i < njobs; i++) {
        J[i].shared.assign(J[i].spec.size(), -1);
        for (size_t b = 0; b < J[i].spec.size(); b++) {
            if (J[i].spec[b].role != PM_IN) continue;
            const char *h = (const char *)jobs[i].host_bufs[b];
            int k = -1;
            for (size_t e = 0; e < sh.size(); e++)
                if (sh[e].host == h) k = (int)e;
            if (k < 0) {
                sh.push_back(SharedIn{h, 0, 0, nullptr});
                k = (int)sh.size() - 1;
            }
            sh[k].bytes = std::max(sh[k].bytes, buf_bytes(J[i].spec[b]));
            sh[k].readers++;
            J[i].shared[b] = k;
        }
    }
    // a region with one reader, or one that any host output of the batch
    // overlaps (its host data may change during the batch), is not shared
    std::vector<bool> keep(sh.size());
    for (size_t e = 0; e < sh.size(); e++) {
        keep[e] = sh[e].readers > 1;
        for (size_t i = 0; i < njobs && keep[e]; i++)
            for (size_t b = 0; b < J[i].spec.size(); b++) {
                if (J[i].spec[b].role != PM_OUT || !jobs[i].host_bufs[b]) continue;
                const char *o0 = (const char *)jobs[i].host_bufs[b], *o1 = o0 + buf_bytes(J[i].spec[b]);
                if (o0 < sh[e].host + sh[e].bytes && sh[e].host < o1) keep[e] = false;
            }
    }
    std::vector<int> renum(sh.size(), -1);
    std::vector<SharedIn> kept;
    for (size_t e = 0; e < sh.size(); e++)
        if (keep[e]) {
            renum[e] = (int)kept.size();
            kept.push_back(sh[e]);
        }
    sh.swap(kept);
    for (auto &j : J)
        for (int &k : j.shared) k = k >= 0 ? renum[k] : -1;
    return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_run_host_batch_bytes(const pm_host_job *jobs, size_t njobs, uint64_t *h2d_bytes, uint64_t *d2h_bytes) {
    std::vector<BatchJob> J;
    std::vector<SharedIn> sh;
    pm_status s = batch_plan("pm_run_host_batch_bytes", jobs, njobs, J, sh);
    if (s) return s;
    uint64_t in = 0, out = 0;
    for (const SharedIn &e : sh) in += e.bytes;
    for (size_t i = 0; i < njobs; i++)
        for (size_t b = 0; b < J[i].spec.size(); b++) {
            if (J[i].spec[b].role == PM_IN && J[i].shared[b] < 0) in += buf_bytes(J[i].spec[b]);
            if (J[i].spec[b].role == PM_OUT && jobs[i].host_bufs[b]) out += buf_bytes(J[i].spec[b]);
        }
    if (h2d_bytes) *h2d_bytes = in;
    if (d2h_bytes) *d2h_bytes = out;
    return PM_OK;
}

pm_status pm_run_host_batch(const pm_host_job *jobs, size_t njobs, const pm_run_opts *opts, void *stream,
                            pm_timing *out, double *copy_ms) {
    if (njobs && (!jobs || !out)) return fail(PM_EINVAL, "pm_run_host_batch: jobs or out is NULL");
    std::vector<BatchJob> J;
    std::vector<SharedIn> sh;
    pm_status s = batch_plan("pm_run_host_batch", jobs, njobs, J, sh);
    if (s) return s;
    if ((s = retain_staging_pool())) return s;
    cudaStream_t cs = (cudaStream_t)stream;
    // does an output of job i overlap an input of job i + 1 in host memory?
    auto clash = [&](size_t i) {
        for (size_t a = 0; a < J[i].spec.size(); a++) {
            if (J[i].spec[a].role != PM_OUT || !jobs[i].host_bufs[a]) continue;
            const char *o0 = (const char *)jobs[i].host_bufs[a];
            const char *o1 = o0 + buf_bytes(J[i].spec[a]);
            for (size_t b = 0; b < J[i + 1].spec.size(); b++) {
                if (J[i + 1].spec[b].role != PM_IN) continue;
                const char *i0 = (const char *)jobs[i + 1].host_bufs[b];
                const char *i1 = i0 + buf_bytes(J[i + 1].spec[b]);
                if (o0 < i1 && i0 < o1) return true;
            }
        }
        return false;
    };
    cudaStream_t up = nullptr, down = nullptr;
    EventPool ev;   // per job: inputs copied, kernels done, outputs copied; then per job: copies begin (in, out)
    pm_status rc = PM_OK;
    if (cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) != cudaSuccess)
        rc = fail(PM_ECUDA, "pm_run_host_batch: stream creation failed");
    if (rc == PM_OK) rc = ev.make(5 * njobs + 2);
    cudaEvent_t *beg = ev.ev.data() + 3 * njobs + 2;   // beg[2 i]: input copies begin, beg[2 i + 1]: output copies
    // Device staging: one slab from the memory pool per batch -- the shared
    // regions at fixed offsets, then two slots for the jobs' own buffers,
    // used by consecutive jobs in turn (a job's inputs never overwrite the
    // slot the previous job's outputs are still being copied from).  One
    // allocation of the same size every batch: the pool reuses it.
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t sh_total = 0, priv_max = 0;
    std::vector<size_t> sh_off(sh.size());
    for (size_t k = 0; k < sh.size(); k++) {
        sh_off[k] = sh_total;
        sh_total += al(sh[k].bytes);
    }
    for (size_t i = 0; i < njobs; i++) {
        size_t priv = 0;
        for (size_t b = 0; b < J[i].spec.size(); b++)
            if (J[i].shared[b] < 0) priv += al(buf_bytes(J[i].spec[b]));
        priv_max = std::max(priv_max, priv);
    }
    unsigned char *slab = nullptr;
    if (rc == PM_OK && njobs) {
        if (alloc_fault_injected() || cudaMallocAsync((void **)&slab, std::max<size_t>(sh_total + 2 * priv_max, 256), up) !=
                                          cudaSuccess) {
            slab = nullptr;
            rc = fail(PM_ENOMEM, "pm_run_host_batch: allocation of %zu staging bytes failed", sh_total + 2 * priv_max);
        }
    }
    double kernels_ms = 0.0;
    for (size_t i = 0; i < njobs && rc == PM_OK; i++) {
        BatchJob &j = J[i];
        cudaEvent_t e_in = ev.ev[3 * i], e_k = ev.ev[3 * i + 1], e_out = ev.ev[3 * i + 2];
        if (i > 0) {
            // inputs of job i after job i-1's kernels (and after its output copy if they alias)
            cudaStreamWaitEvent(up, ev.ev[3 * (i - 1) + 1], 0);
            if (clash(i - 1)) cudaStreamWaitEvent(up, ev.ev[3 * (i - 1) + 2], 0);
        }
        if (i > 1) cudaStreamWaitEvent(up, ev.ev[3 * (i - 2) + 2], 0);   // job i-2's outputs left this slot
        if (i == 0) cudaEventRecord(ev.ev[3 * njobs], up);
        cudaEventRecord(beg[2 * i], up);
        if (i == 0)   // every shared region in one burst of back-to-back copies, before any kernel
            for (size_t k = 0; k < sh.size() && rc == PM_OK; k++) {
                sh[k].dev = slab + sh_off[k];
                if (cudaMemcpyAsync(sh[k].dev, sh[k].host, sh[k].bytes, cudaMemcpyHostToDevice, up) != cudaSuccess)
                    rc = fail(PM_ECUDA, "pm_run_host_batch: host-to-device copy of shared region %zu failed", k);
            }
        std::vector<void *> bufs(j.spec.size(), nullptr);
        unsigned char *slot = slab + sh_total + (i % 2) * priv_max;
        for (size_t b = 0; b < j.spec.size() && rc == PM_OK; b++) {
            const int k = j.shared[b];
            if (k >= 0) {   // a shared input, already on the device
                bufs[b] = sh[k].dev;
                continue;
            }
            const size_t bytes = buf_bytes(j.spec[b]);
            bufs[b] = slot;
            slot += al(bytes);
            if (j.spec[b].role == PM_IN &&
                cudaMemcpyAsync(bufs[b], jobs[i].host_bufs[b], bytes, cudaMemcpyHostToDevice, up) != cudaSuccess)
                rc = fail(PM_ECUDA, "pm_run_host_batch: job %zu: host-to-device copy failed", i);
        }
        if (rc != PM_OK) break;
        cudaEventRecord(e_in, up);
        cudaStreamWaitEvent(cs, e_in, 0);
        if (i > 0) cudaStreamWaitEvent(cs, ev.ev[3 * (i - 1) + 2], 0);   // no kernel under a copy
        pm_timing t{};
        rc = timed(j.kp, bufs.data(), bufs.size(), opts, stream, nullptr, &t);
        if (rc != PM_OK) {
            const std::string why = pm_last_error();
            fail(rc, "pm_run_host_batch: job %zu (%s): %s", i, j.kp.def->name, why.c_str());
            break;
        }
        out[i] = t;
        kernels_ms += t.mean_ms * t.n_trials;
        cudaEventRecord(e_k, cs);
        cudaStreamWaitEvent(down, e_k, 0);
        cudaEventRecord(beg[2 * i + 1], down);
        for (size_t b = 0; b < j.spec.size() && rc == PM_OK; b++)
            if (j.spec[b].role == PM_OUT && jobs[i].host_bufs[b] &&
                cudaMemcpyAsync(jobs[i].host_bufs[b], bufs[b], buf_bytes(j.spec[b]), cudaMemcpyDeviceToHost, down) !=
                    cudaSuccess)
                rc = fail(PM_ECUDA, "pm_run_host_batch: job %zu: device-to-host copy failed", i);
        cudaEventRecord(e_out, down);
    }
    if (up) cudaStreamSynchronize(up);
    if (down) {
        if (rc == PM_OK && njobs) cudaEventRecord(ev.ev[3 * njobs + 1], down);
        cudaStreamSynchronize(down);
    }
    cudaStreamSynchronize(cs);
    if (slab) {   // every stream that used it has drained
        cudaFreeAsync(slab, cs);
        cudaStreamSynchronize(cs);
    }
    if (rc == PM_OK && copy_ms && njobs) {
        // the copies' own device time: each job's input copies (after it may
        // start) and output copies, summed; the time between them (kernels,
        // host work between jobs) is not included
        double tot = 0.0;
        for (size_t i = 0; i < njobs; i++) {
            float a = 0.0f, b = 0.0f;
            cudaEventElapsedTime(&a, beg[2 * i], ev.ev[3 * i]);
            cudaEventElapsedTime(&b, beg[2 * i + 1], ev.ev[3 * i + 2]);
            tot += (double)a + (double)b;
        }
        *copy_ms = tot;
    }
    (void)kernels_ms;
    if (up) cudaStreamDestroy(up);
    if (down) cudaStreamDestroy(down);
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------- load latency probe
// A pointer chase over 128-byte lines: line i holds the index of line
// (i + stride) mod nlines, stride coprime with nlines (every line visited
// once per cycle), read with L1-bypassing loads by one thread, so each hop
// waits for the previous one: the unloaded latency of the level that holds
// the buffer (HBM for a buffer far larger than L2, L2 for a small one).
namespace pm {
namespace {
__global__ void k_chase_init(uint32_t *next, uint32_t nlines, uint32_t stride) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nlines; i += (size_t)gridDim.x * blockDim.x)
        next[i * 32] = (uint32_t)((i + stride) % nlines);
}
__global__ void k_chase(const uint32_t *__restrict__ next, uint32_t nlines, uint32_t hops, uint32_t *sink) {
    uint32_t p = 0;
    for (uint32_t h = 0; h < hops; h++) {
        p = __ldcg(next + (size_t)p * 32);
        if (p >= nlines) break;   // cannot happen for an initialised chain; keeps every read in bounds
    }
    *sink = p;
}
uint64_t gcd_u64(uint64_t a, uint64_t b) {
    while (b) { const uint64_t t = a % b; a = b; b = t; }
    return a;
}
}  // namespace
}  // namespace pm

extern "C" pm_status pm_probe_latency(void *buf, size_t bytes, int32_t hops, double *ns_per_hop, void *stream) {
    using namespace pm;
    if (!buf || !ns_per_hop || hops < 1 || bytes < 256 || bytes / 128 > 0xffffffffull || (uintptr_t)buf % 128)
        return fail(PM_EINVAL, "pm_probe_latency: need a 128-byte aligned buffer of 256 bytes .. 512 GiB and hops >= 1");
    const uint32_t nlines = (uint32_t)(bytes / 128);
    uint64_t s = (uint64_t)(nlines * 0.6180339887) | 1u;
    while (s < 2 || gcd_u64(s, nlines) != 1) s += 1;
    s %= nlines;
    if (s == 0) s = 1;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *next = (uint32_t *)buf;
    k_chase_init<<<1216, 256, 0, st>>>(next, nlines, (uint32_t)s);
    PM_CUDA_TRY(cudaGetLastError());
    // the sink: the word after the first line's index (never an index slot)
    uint32_t *sink = next + 1;
    EventPool ev;
    pm_status rc = ev.make(2);
    if (rc) return rc;
    k_chase<<<1, 1, 0, st>>>(next, nlines, (uint32_t)std::min<int32_t>(hops, 64), sink);   // warm-up
    PM_CUDA_TRY(cudaEventRecord(ev.ev[0], st));
    k_chase<<<1, 1, 0, st>>>(next, nlines, (uint32_t)hops, sink);
    PM_CUDA_TRY(cudaEventRecord(ev.ev[1], st));
    PM_CUDA_TRY(cudaEventSynchronize(ev.ev[1]));
    PM_CUDA_TRY(cudaGetLastError());
    float ms = 0.0f;
    PM_CUDA_TRY(cudaEventElapsedTime(&ms, ev.ev[0], ev.ev[1]));
    *ns_per_hop = (double)ms * 1e6 / hops;
    return PM_OK;
}
