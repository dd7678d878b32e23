// C ABI plumbing: error buffer, kernel registry, parameter parsing, pm_counts,
// pm_kernel_buffers.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <limits>

#include "pm_internal.h"

namespace pm {

static thread_local char g_err[1024];

pm_status fail(pm_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}
void clear_error() { g_err[0] = 0; }

// allocation failure injection (pm_test_fail_allocation): countdown per thread
static thread_local int g_fail_alloc = 0;
void set_fail_allocation(int n) { g_fail_alloc = n; }
bool alloc_fault_injected() {
    if (g_fail_alloc <= 0) return false;
    return --g_fail_alloc == 0;
}

static constexpr double REQ = std::numeric_limits<double>::quiet_NaN();

// Parameter lists of each kernel family.  Integer unless noted.
#define P_STREAM {"dtype", "vec", "N", "s", "L", "shape", "W", nullptr}, {0, 0, REQ, 1, 1, 0, 16, 0}, \
                 {1, 1, 1, 1, 1, 1, 1, 1}
#define P_FMA {"dtype", "op", "F", "G", nullptr}, {0, 2, REQ, REQ}, {1, 1, 1, 1}
#define P_SMEM {"R", "sync", "G", nullptr}, {REQ, 0, REQ}, {1, 1, 1}
#define P_BAR {"B", "G", nullptr}, {REQ, REQ}, {1, 1}
#define P_OVL {"m", "N", nullptr}, {REQ, REQ}, {1, 1}
#define P_EMPTY {"G", nullptr}, {REQ}, {1}
#define P_MM {"n", nullptr}, {REQ}, {1}
#define P_DG {"Np", "Nel", "L0", "L1", nullptr}, {REQ, REQ, 16, 16}, {1, 1, 1, 1}
#define P_FD {"n", "c0", "c1", nullptr}, {REQ, -4.0, 1.0}, {1, 0, 0}
#define P_SIMT {"n", "BM", "BN", "BK", nullptr}, {REQ, 128, 128, 32}, {1, 1, 1, 1}
#define P_SMEM2D {"R", "T", "G", nullptr}, {REQ, 16, REQ}, {1, 1, 1}
#define P_TC {"n", "pipe", nullptr}, {REQ, 1}, {1, 1}
#define P_TCW {"n", nullptr}, {REQ}, {1}
#define P_DGT {"Np", "Nel", nullptr}, {REQ, REQ}, {1, 1}
#define P_DGC {"Np", "Nel", "P", "A", nullptr}, {REQ, REQ, 0, -1}, {1, 1, 1, 1}
#define P_FDB {"n", "BX", "BY", "c0", "c1", "V", nullptr}, {REQ, 64, 8, -4.0, 1.0, 4}, {1, 1, 1, 0, 0, 1}

static const KernelDef KDEFS[] = {
    {"stream", FAM_STREAM, 0, P_STREAM},
    {"fma", FAM_FMA, 0, P_FMA},
    {"smem", FAM_SMEM, 0, P_SMEM},
    {"barrier", FAM_BARRIER, 0, P_BAR},
    {"overlap", FAM_OVERLAP, 0, P_OVL},
    {"empty", FAM_EMPTY, 0, P_EMPTY},
    {"mm_pf", FAM_MM, 0, P_MM},
    {"mm_nopf", FAM_MM, 1, P_MM},
    {"mm_pf_a", FAM_MM, 2, P_MM},
    {"mm_pf_b", FAM_MM, 3, P_MM},
    {"mm_nopf_a", FAM_MM, 4, P_MM},
    {"mm_nopf_b", FAM_MM, 5, P_MM},
    {"dg_nopf", FAM_DG, 0, P_DG},
    {"dg_dmpf", FAM_DG, 1, P_DG},
    {"dg_nopf_u", FAM_DG, 2, P_DG},
    {"dg_nopf_dm", FAM_DG, 3, P_DG},
    {"dg_dmpf_u", FAM_DG, 4, P_DG},
    {"dg_dmpf_dm", FAM_DG, 5, P_DG},
    {"dg_res", FAM_DG, 6, P_DG},
    {"fd_tile", FAM_FD, 0, P_FD},
    {"fd_direct", FAM_FD, 1, P_FD},
    {"fd_tile_u", FAM_FD, 2, P_FD},
    {"fd_tile_res", FAM_FD, 3, P_FD},
    {"fd_direct_u", FAM_FD, 4, P_FD},
    {"fd_direct_res", FAM_FD, 5, P_FD},
    {"mm_simt", FAM_SIMT, 0, P_SIMT},
    {"mm_tc", FAM_TC, 0, P_TC},
    {"fd_block", FAM_FDB, 0, P_FDB},
    {"fd_tile18", FAM_FD, 6, P_FD},
    {"fd_tile18_u", FAM_FD, 7, P_FD},
    {"fd_tile18_res", FAM_FD, 8, P_FD},
    {"dg_upf", FAM_DG, 7, P_DG},
    {"dg_dmpft", FAM_DG, 8, P_DG},
    {"dg_upf_u", FAM_DG, 9, P_DG},
    {"dg_dmpft_u", FAM_DG, 10, P_DG},
    {"dg_dmpft_res", FAM_DG, 11, P_DG},
    {"smem2d", FAM_SMEM2D, 0, P_SMEM2D},
    {"mm_tc256", FAM_TC, 1, P_TCW},
    {"dg_tile", FAM_DGT, 0, P_DGT},
    {"dg_tc", FAM_DGC, 0, P_DGC},
};

const KernelDef *kernel_def(int32_t id) {
    if (id < 0 || id >= (int32_t)(sizeof KDEFS / sizeof KDEFS[0])) return nullptr;
    return &KDEFS[id];
}
int32_t kernel_total() { return (int32_t)(sizeof KDEFS / sizeof KDEFS[0]); }

pm_status parse_params(int32_t kernel, const pm_param *p, size_t np, KP *out) {
    const KernelDef *d = kernel_def(kernel);
    if (!d) return fail(PM_EUNKNOWN_KERNEL, "unknown kernel id %d", kernel);
    if (np && !p) return fail(PM_EINVAL, "params is NULL but np = %zu", np);
    KP kp;
    kp.def = d;
    int n = 0;
    while (n < kMaxParams && d->pnames[n]) n++;
    bool seen[kMaxParams] = {false};
    for (size_t a = 0; a < np; a++) {
        if (!p[a].key) return fail(PM_EINVAL, "parameter %zu has a NULL key", a);
        int k = -1;
        for (int b = 0; b < n; b++)
            if (!strcmp(p[a].key, d->pnames[b])) k = b;
        if (k < 0) return fail(PM_EINVAL, "kernel %s has no parameter '%s'", d->name, p[a].key);
        double v = p[a].value;
        if (!std::isfinite(v)) return fail(PM_EINVAL, "%s: parameter %s is not finite", d->name, p[a].key);
        if (d->pinteger[k] && (v != std::floor(v) || std::fabs(v) > 9.0e15))
            return fail(PM_EINVAL, "%s: parameter %s must be an integer (got %g)", d->name, p[a].key, v);
        kp.v[k] = v;
        seen[k] = true;
    }
    for (int b = 0; b < n; b++)
        if (!seen[b]) {
            if (std::isnan(d->pdefault[b]))
                return fail(PM_EINVAL, "%s: missing required parameter '%s'", d->name, d->pnames[b]);
            kp.v[b] = d->pdefault[b];
        }
    *out = kp;
    return PM_OK;
}

static void afr_text(uint64_t acc, uint64_t foot, char *buf, size_t cap) {
    uint64_t a = acc, b = foot;
    while (b) { uint64_t t = a % b; a = b; b = t; }
    uint64_t g = a ? a : 1;
    if (foot / g == 1) snprintf(buf, cap, "%llu", (unsigned long long)(acc / g));
    else snprintf(buf, cap, "%llu/%llu", (unsigned long long)(acc / g), (unsigned long long)(foot / g));
}

void canonical_name(pm_feature &f) {
    switch (f.kind) {
    case PM_FEAT_OP:
        snprintf(f.name, sizeof f.name, "f_op_%s_%s", f.dtype, f.op);
        break;
    case PM_FEAT_MEM: {
        char ls[96] = "", gs[96] = "", afr[48];
        size_t o = 0;
        for (int a = 0; a < f.nl; a++)
            o += snprintf(ls + o, sizeof ls - o, "%s%d:%lld", a ? ";" : "", a, (long long)f.lstride[a]);
        o = 0;
        for (int a = 0; a < f.ng; a++)
            o += snprintf(gs + o, sizeof gs - o, "%s%d:%lld", a ? ";" : "", a, (long long)f.gstride[a]);
        afr_text(f.accesses, f.footprint, afr, sizeof afr);
        snprintf(f.name, sizeof f.name, "f_mem_access_tag:%s_%s_%s_%s_lstrides:{%s}_gstrides:{%s}_afr:%s", f.tag,
                 f.mem ? "local" : "global", f.dtype, f.dir ? "store" : "load", ls, gs, afr);
        break;
    }
    case PM_FEAT_SYNC: snprintf(f.name, sizeof f.name, "f_sync_barrier_local"); break;
    case PM_FEAT_GROUPS: snprintf(f.name, sizeof f.name, "f_thread_groups"); break;
    case PM_FEAT_LAUNCH: snprintf(f.name, sizeof f.name, "f_sync_kernel_launch"); break;
    }
}

}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_test_fail_allocation(int32_t n) {
    if (n < 0) return pm::fail(PM_EINVAL, "pm_test_fail_allocation: n must be >= 0");
    pm::set_fail_allocation(n);
    return PM_OK;
}

const char *pm_last_error(void) { return g_err; }

pm_status pm_kernel_lookup(const char *name, int32_t *kernel) {
    if (!name || !kernel) return fail(PM_EINVAL, "pm_kernel_lookup: NULL argument");
    for (int32_t i = 0; i < kernel_total(); i++)
        if (!strcmp(KDEFS[i].name, name)) {
            *kernel = i;
            return PM_OK;
        }
    return fail(PM_EUNKNOWN_KERNEL, "unknown kernel '%s'", name);
}

pm_status pm_kernel_count(int32_t *n) {
    if (!n) return fail(PM_EINVAL, "pm_kernel_count: NULL argument");
    *n = kernel_total();
    return PM_OK;
}

pm_status pm_kernel_name(int32_t kernel, const char **name) {
    if (!name) return fail(PM_EINVAL, "pm_kernel_name: NULL argument");
    const KernelDef *d = kernel_def(kernel);
    if (!d) return fail(PM_EUNKNOWN_KERNEL, "unknown kernel id %d", kernel);
    *name = d->name;
    return PM_OK;
}

pm_status pm_counts(int32_t kernel, const pm_param *p, size_t np, pm_feature *out, size_t cap, size_t *n_out) {
    if (!n_out) return fail(PM_EINVAL, "pm_counts: n_out is NULL");
    if (cap && !out) return fail(PM_EINVAL, "pm_counts: out is NULL but cap = %zu", cap);
    KP kp;
    pm_status s = parse_params(kernel, p, np, &kp);
    if (s) return s;
    std::vector<pm_feature> v;
    s = counts(kp, v);
    if (s) return s;
    *n_out = v.size();
    if (v.size() > cap) return fail(PM_ECAP, "pm_counts: %zu records needed, cap is %zu", v.size(), cap);
    for (size_t i = 0; i < v.size(); i++) {
        canonical_name(v[i]);
        out[i] = v[i];
    }
    return PM_OK;
}

pm_status pm_kernel_buffers(int32_t kernel, const pm_param *p, size_t np, pm_buffer *out, size_t cap,
                            size_t *n_out) {
    if (!n_out) return fail(PM_EINVAL, "pm_kernel_buffers: n_out is NULL");
    if (cap && !out) return fail(PM_EINVAL, "pm_kernel_buffers: out is NULL but cap = %zu", cap);
    KP kp;
    pm_status s = parse_params(kernel, p, np, &kp);
    if (s) return s;
    if ((s = validate(kp))) return s;
    std::vector<BufSpec> v;
    if ((s = buffers(kp, v))) return s;
    *n_out = v.size();
    if (v.size() > cap) return fail(PM_ECAP, "pm_kernel_buffers: %zu buffers, cap is %zu", v.size(), cap);
    for (size_t i = 0; i < v.size(); i++) {
        memset(&out[i], 0, sizeof out[i]);
        snprintf(out[i].name, sizeof out[i].name, "%s", v[i].name);
        out[i].dtype = v[i].dtype;
        out[i].role = v[i].role;
        out[i].elems = v[i].elems;
    }
    return PM_OK;
}

}  // extern "C"
