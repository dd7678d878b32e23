// Internal declarations shared by the translation units of libpm.so.
#pragma once
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "pm.h"

namespace pm {

// ---- errors -------------------------------------------------------------
pm_status fail(pm_status s, const char *fmt, ...);
void clear_error();
bool alloc_fault_injected();   // pm_test_fail_allocation countdown (true: fail this allocation)
// Raise the release threshold of the current device's default memory pool to
// the maximum (once per device), so memory freed with cudaFreeAsync stays
// reserved for the next cudaMallocAsync instead of being unmapped.
pm_status retain_staging_pool();
void set_fail_allocation(int n);

// An allocation: PM_ENOMEM when it is refused for lack of memory (or a test
// injected the failure, see pm_test_fail_allocation), PM_ECUDA otherwise.
#define PM_ALLOC_TRY(expr)                                                                  \
    do {                                                                                    \
        if (::pm::alloc_fault_injected())                                                   \
            return ::pm::fail(PM_ENOMEM, "%s: allocation failed (injected)", #expr);        \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::pm::fail(e_ == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA, "%s: %s (%s:%d)", \
                              #expr, cudaGetErrorString(e_), __FILE__, __LINE__);           \
    } while (0)

#define PM_CUDA_TRY(expr)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::pm::fail(PM_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),    \
                              __FILE__, __LINE__);                                          \
    } while (0)

// ---- kernel registry ------------------------------------------------------
enum Family { FAM_STREAM, FAM_FMA, FAM_SMEM, FAM_BARRIER, FAM_OVERLAP, FAM_EMPTY, FAM_MM, FAM_DG, FAM_FD, FAM_SIMT, FAM_TC, FAM_FDB,
              FAM_SMEM2D, FAM_DGT, FAM_DGC };

constexpr int kMaxParams = 8;

struct KernelDef {
    const char *name;
    Family fam;
    int variant;
    const char *pnames[kMaxParams];  // parameter names in order (nullptr-terminated)
    double pdefault[kMaxParams];     // NaN = required
    bool pinteger[kMaxParams];
};

const KernelDef *kernel_def(int32_t id);
int32_t kernel_total();

// Parsed kernel parameters (values by position in KernelDef::pnames).
struct KP {
    const KernelDef *def = nullptr;
    double v[kMaxParams] = {0};
    int64_t i(int k) const { return (int64_t)v[k]; }
};

pm_status parse_params(int32_t kernel, const pm_param *p, size_t np, KP *out);

// ---- counts (pm_counts.cpp) ---------------------------------------------------
// Validates the parameters for the family and fills feature records.
pm_status counts(const KP &kp, std::vector<pm_feature> &out);
// Validation only (shared by launch paths).
pm_status validate(const KP &kp);

// ---- buffers and launches (pm_suite.cu, pm_modeled.cu) -------------------------
struct BufSpec {
    const char *name;
    int dtype;
    int role;
    uint64_t elems;
};
pm_status buffers(const KP &kp, std::vector<BufSpec> &out);
// Launch query: while a LaunchQuery is installed on the calling thread, the
// launch helpers record the kernel they would launch (attributes, occupancy,
// launch shape) instead of launching it.  Used by pm_kernel_resources.
struct LaunchQuery {
    pm_resources *out;
    int hits;
    pm_status status;
};
extern thread_local LaunchQuery *g_launch_query;
// Returns true when the launch must be skipped (a query is installed).
bool launch_query_hook(const void *fn, unsigned gx, unsigned gy, unsigned gz, unsigned bx, unsigned by, unsigned bz,
                       size_t smem);

#ifdef __CUDACC__
template <typename... P, typename... A>
inline void launch_k(void (*k)(P...), dim3 g, dim3 b, size_t smem, cudaStream_t st, A... a) {
    if (launch_query_hook((const void *)k, g.x, g.y, g.z, b.x, b.y, b.z, smem)) return;
    k<<<g, b, smem, st>>>(static_cast<P>(a)...);
}
#endif

pm_status launch_suite(const KP &kp, void *const *bufs, void *stream);
pm_status launch_modeled(const KP &kp, void *const *bufs, void *stream);
pm_status launch_tiles(const KP &kp, void *const *bufs, void *stream);
pm_status launch_tc(const KP &kp, void *const *bufs, void *stream);
pm_status tc_check_timeout();
pm_status fdb_check_timeout();
pm_status dgt_check_timeout();
pm_status launch_dgc(const KP &kp, void *const *bufs, void *stream);
pm_status dgc_check_timeout();
// dg_tc geometry shared by the launch and the counts: m per CTA, CTAs per SM,
// shared-memory stages and output staging buffers of the u operand's form
// (the stages and buffers of A = 0; A = 1 has 4 raw stages when Np % 4 == 0
// and 2 staging buffers)
struct DgcShape {
    int ms, r, st, ob;
};
DgcShape dgc_geometry(int Np, int A);
int dgc_resolve_a(int Np, int A);                      // -1: the library's choice for Np
int dgc_resolve_p(int Np, int64_t Nel, int A, int P);  // 0: one wave of a GB300
// 2-D tensor map (TMA descriptor) over a row-major matrix; `map` must point
// to a CUtensorMap (64-byte aligned, 128 bytes).
pm_status tensor_map_2d(struct CUtensorMap_st *map, int bf16, const void *ptr, uint64_t cols, uint64_t rows,
                        uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows, int swizzle128);

// ---- feature records helper --------------------------------------------------
void canonical_name(pm_feature &f);

}  // namespace pm
