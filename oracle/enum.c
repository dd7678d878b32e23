/*
 * ORACLE -- test infrastructure only.  Only tests/, __graft_entry__.smoke()
 * and the cpu_baseline leg of bench.py may load this code.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Brute-force kernel statistics by literal enumeration of the loop domain
 * (Section "Gathering Kernel Statistics", Algorithm 1 and Algorithm 2), plus
 * plain reference outputs of every kernel (FP64 sums, or bit-exact FP32/FP64
 * replays where the kernel's operation order is fixed by its definition).
 *
 * How a kernel is described here: a walker function literally executes the
 * kernel's loop nest for ONE work-item (group id g[3], local id l[3]) and
 * reports each executed statement instance via X(ctx, stmt, loopvars) and
 * each barrier via BAR(ctx).  Each statement lists its floating point
 * operations and its memory access sites; each site has an index function of
 * (g, l, loopvars).  From these the enumerator computes:
 *   - per statement: sub-group (SG) instance counts, i.e. how many distinct
 *     (statement, loop-variable) instances the 32 lanes of a sub-group execute
 *     (on-chip work is counted per SG, Section "Gathering Kernel Statistics");
 *   - per access site: work-item (WI) access count, SG count, local/global
 *     strides as finite differences of the index along each thread axis
 *     (checked constant over the whole domain = affinity check), the stride
 *     along the innermost enclosing sequential loop (Table "ab_pattern"), and
 *     the footprint = number of distinct indices touched (Algorithm 2, applied
 *     per access site);
 *   - barriers encountered by a single work-item (Section "Gathering Kernel
 *     Statistics", barrier counting), work-group count, one kernel launch.
 * Sub-groups are lanes 32q..32q+31 of the linear id lid0 + L0*lid1 + L0*L1*lid2.
 *
 * Every function in this file is pinned by tests in tests/test_oracle_*.py
 * against closed forms and values the paper fixes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <stdio.h>

#define MAXSITE 24
#define MAXSTMT 24
#define MAXLOOP 3
#define SGSIZE 32

enum { MEM_GLOBAL = 0, MEM_LOCAL = 1 };
enum { DIR_LOAD = 0, DIR_STORE = 1 };
enum { DT_F32 = 0, DT_F64 = 1, DT_BF16 = 2, DT_TF32 = 3 };

typedef struct ctx ctx;
typedef long long (*idx_fn)(const ctx *c, const long long *g, const long long *l, const long long *lv);

typedef struct {
    char tag[24];
    int mem, dir, dsize;
    char dtype[16];
    idx_fn idx;
} site_t;

typedef struct {
    int nloop;
    int n_add, n_mul, n_madd;   /* scalar floating point ops per instance */
    int dt;                     /* DT_F32 / DT_F64 */
    int nsite;
    int site[8];
} stmt_t;

/* open-addressing set of non-negative 64-bit keys (-1 = empty) */
typedef struct {
    long long *k;
    size_t cap, n;
} kset;

static void ks_init(kset *s, size_t cap) {
    s->cap = cap; s->n = 0;
    s->k = (long long *)malloc(cap * sizeof(long long));
    for (size_t i = 0; i < cap; i++) s->k[i] = -1;
}
static void ks_free(kset *s) { free(s->k); s->k = NULL; s->cap = s->n = 0; }
static void ks_clear(kset *s) { for (size_t i = 0; i < s->cap; i++) s->k[i] = -1; s->n = 0; }
static size_t ks_hash(long long x) {
    unsigned long long z = (unsigned long long)x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return (size_t)(z ^ (z >> 31));
}
static int ks_insert(kset *s, long long key);
static void ks_grow(kset *s) {
    kset t; ks_init(&t, s->cap * 2);
    for (size_t i = 0; i < s->cap; i++) if (s->k[i] >= 0) ks_insert(&t, s->k[i]);
    free(s->k); *s = t;
}
/* returns 1 if newly inserted */
static int ks_insert(kset *s, long long key) {
    if ((s->n + 1) * 2 > s->cap) ks_grow(s);
    size_t m = s->cap - 1, h = ks_hash(key) & m;
    while (s->k[h] >= 0) {
        if (s->k[h] == key) return 0;
        h = (h + 1) & m;
    }
    s->k[h] = key; s->n++;
    return 1;
}

typedef struct {
    unsigned long long wi, sg;
    kset foot;
    long long lstr[3], gstr[3], loopstr;
    int have_str, affine, have_loop;
} site_stat;

struct ctx {
    long long P[8];          /* kernel parameters (meaning per kernel) */
    long long D[8];          /* derived constants */
    long long grid[3], wg[3];
    int nsite, nstmt;
    site_t site[MAXSITE];
    stmt_t stmt[MAXSTMT];
    void (*walk)(ctx *c);
    /* current work-item */
    long long g[3], l[3];
    /* accumulators */
    site_stat ss[MAXSITE];
    unsigned long long op_wi[4][3], op_sg[4][3];  /* [dtype][add,mul,madd] */
    unsigned long long stmt_sg[MAXSTMT], stmt_wi[MAXSTMT];
    long long bar_cur, bar_min, bar_max;
    kset sgset;              /* distinct statement instances of the current SG */
    int err;
    /* work removal (Algorithm 3): parent statement -> its twin statements */
    int twin, tdest;
    int tmap_n[MAXSTMT], tmap[MAXSTMT][8];
};

static int add_site(ctx *c, const char *tag, int mem, int dir, const char *dtype, int dsize, idx_fn f) {
    site_t *s = &c->site[c->nsite];
    memset(s, 0, sizeof *s);
    strncpy(s->tag, tag, sizeof s->tag - 1);
    strncpy(s->dtype, dtype, sizeof s->dtype - 1);
    s->mem = mem; s->dir = dir; s->dsize = dsize; s->idx = f;
    return c->nsite++;
}
static int add_stmt(ctx *c, int nloop, int dt, int nadd, int nmul, int nmadd) {
    stmt_t *s = &c->stmt[c->nstmt];
    memset(s, 0, sizeof *s);
    s->nloop = nloop; s->dt = dt; s->n_add = nadd; s->n_mul = nmul; s->n_madd = nmadd;
    return c->nstmt++;
}
static void stmt_site(ctx *c, int st, int site) { stmt_t *s = &c->stmt[st]; s->site[s->nsite++] = site; }

static void X_exec(ctx *c, int st, const long long *lv);
/* one executed statement instance of the current work-item; in work-removal
 * mode the parent statement is replaced by the statements derived from it */
static void X(ctx *c, int st, const long long *lv) {
    if (!c->twin) { X_exec(c, st, lv); return; }
    for (int k = 0; k < c->tmap_n[st]; k++) X_exec(c, c->tmap[st][k], lv);
}
static void X_exec(ctx *c, int st, const long long *lv) {
    const stmt_t *S = &c->stmt[st];
    long long key = st;
    for (int i = 0; i < S->nloop; i++) {
        if (lv[i] < 0 || lv[i] >= (1LL << 19)) { c->err = 1; return; }
        key = key | (lv[i] << (6 + 19 * i));
    }
    int fresh = ks_insert(&c->sgset, key);
    c->stmt_wi[st]++;
    c->op_wi[S->dt][0] += S->n_add; c->op_wi[S->dt][1] += S->n_mul; c->op_wi[S->dt][2] += S->n_madd;
    if (fresh) {
        c->stmt_sg[st]++;
        c->op_sg[S->dt][0] += S->n_add; c->op_sg[S->dt][1] += S->n_mul; c->op_sg[S->dt][2] += S->n_madd;
    }
    for (int a = 0; a < S->nsite; a++) {
        int si = S->site[a];
        site_stat *t = &c->ss[si];
        idx_fn f = c->site[si].idx;
        long long base = f(c, c->g, c->l, lv);
        if (base < 0) { c->err = 2; return; }
        t->wi++;
        if (fresh) t->sg++;
        ks_insert(&t->foot, base);
        long long ls[3], gs[3], lps = 0;
        for (int ax = 0; ax < 3; ax++) {
            long long l2[3] = {c->l[0], c->l[1], c->l[2]};
            long long g2[3] = {c->g[0], c->g[1], c->g[2]};
            l2[ax] += 1; g2[ax] += 1;
            ls[ax] = f(c, c->g, l2, lv) - base;
            gs[ax] = f(c, g2, c->l, lv) - base;
        }
        if (S->nloop > 0) {
            long long lv2[MAXLOOP];
            for (int i = 0; i < S->nloop; i++) lv2[i] = lv[i];
            lv2[S->nloop - 1] += 1;
            lps = f(c, c->g, c->l, lv2) - base;
        }
        if (!t->have_str) {
            for (int ax = 0; ax < 3; ax++) { t->lstr[ax] = ls[ax]; t->gstr[ax] = gs[ax]; }
            t->loopstr = lps; t->have_loop = S->nloop > 0;
            t->have_str = 1; t->affine = 1;
        } else {
            for (int ax = 0; ax < 3; ax++)
                if (t->lstr[ax] != ls[ax] || t->gstr[ax] != gs[ax]) t->affine = 0;
            if (t->loopstr != lps) t->affine = 0;
        }
    }
}
static void BAR(ctx *c) { if (!c->twin) c->bar_cur++; }   /* work removal drops barriers with the local memory */

/* ---------------------------------------------------------------- helpers */
#define G0 (g[0])
#define G1 (g[1])
#define L0_ (l[0])
#define L1_ (l[1])
static long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

/* ======================================================================
 * Calibration suite (Section "Measurement Kernel Design")
 * ====================================================================== */

/* stream: result[pattern] = sum_{a<L} in_a[pattern]   (global memory access
 * measurement kernel, AFR 1).  P = {dtype, vec, N, s, L, shape, W}.
 * vec: 0 scalar, 1 16-byte vectors (float32x4 / float64x2).
 * shape 0: 1-D work-group of 256, index = s*lid0 + gid0 + 256*s*gid1,
 *          grid (s, M/(256 s)), M = N/w vectors.
 * shape 1: 16x16 work-group over a row-major M/W x W array:
 *          index = lid0 + W*lid1 + 16*gid0 + 16*W*gid1, grid (W/16, M/(16W)). */
static long long ix_stream(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv;
    if (c->P[5] == 0) { long long s = c->P[3]; return s * L0_ + G0 + 256 * s * G1; }
    long long W = c->P[6];
    return L0_ + W * L1_ + 16 * G0 + 16 * W * G1;
}
static void walk_stream(ctx *c) { X(c, 0, NULL); }
static int setup_stream(ctx *c) {
    long long dt = c->P[0], vec = c->P[1], N = c->P[2], s = c->P[3], L = c->P[4], shape = c->P[5], W = c->P[6];
    if (dt < 0 || dt > 1 || vec < 0 || vec > 1 || L < 1 || L > 4 || N <= 0) return -1;
    long long w = vec ? (dt == DT_F32 ? 4 : 2) : 1;
    if (N % w) return -1;
    long long M = N / w;
    const char *dn = dt == DT_F32 ? (vec ? "float32x4" : "float32") : (vec ? "float64x2" : "float64");
    int ds = vec ? 16 : (dt == DT_F32 ? 4 : 8);
    if (shape == 0) {
        if (s < 1 || M % (256 * s)) return -1;
        c->grid[0] = s; c->grid[1] = M / (256 * s); c->grid[2] = 1;
        c->wg[0] = 256; c->wg[1] = 1; c->wg[2] = 1;
    } else if (shape == 1) {
        if (W < 16 || W % 16 || M % (16 * W)) return -1;
        c->grid[0] = W / 16; c->grid[1] = M / (16 * W); c->grid[2] = 1;
        c->wg[0] = 16; c->wg[1] = 16; c->wg[2] = 1;
    } else return -1;
    int st = add_stmt(c, 0, (int)dt, (int)((L - 1) * w), 0, 0);
    static const char *nm[4] = {"in0", "in1", "in2", "in3"};
    for (int a = 0; a < L; a++) stmt_site(c, st, add_site(c, nm[a], MEM_GLOBAL, DIR_LOAD, dn, ds, ix_stream));
    stmt_site(c, st, add_site(c, "out", MEM_GLOBAL, DIR_STORE, dn, ds, ix_stream));
    c->walk = walk_stream;
    return 0;
}

/* arithmetic kernel: 32 private variables per work-item, each updated F/32
 * times with the target operation; no update reads a variable written by the
 * four most recent updates (each variable only reads itself).  P = {dtype, op, F, G}
 * op 0 add, 1 mul, 2 madd.  Work-group 256, G groups. */
static long long ix_lin(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)c; (void)lv; return 256 * G0 + L0_;
}
static void walk_fma(ctx *c) {
    long long lv[2];
    X(c, 0, NULL);                                       /* u = seed[gtid] */
    for (lv[0] = 0; lv[0] < 32; lv[0]++) X(c, 1, lv);    /* x_t = u + c_t */
    long long R = c->P[2] / 32;
    for (lv[0] = 0; lv[0] < R; lv[0]++)
        for (lv[1] = 0; lv[1] < 32; lv[1]++) X(c, 2, lv); /* x_t = op(x_t) */
    for (lv[0] = 1; lv[0] < 32; lv[0]++) X(c, 3, lv);    /* s = s + x_t */
    X(c, 4, NULL);                                       /* out[gtid] = s */
}
static int setup_fma(ctx *c) {
    long long dt = c->P[0], op = c->P[1], F = c->P[2], G = c->P[3];
    if (dt < 0 || dt > 1 || op < 0 || op > 2 || F < 32 || F % 32 || G < 1) return -1;
    const char *dn = dt == DT_F32 ? "float32" : "float64";
    int ds = dt == DT_F32 ? 4 : 8;
    c->grid[0] = G; c->grid[1] = 1; c->grid[2] = 1;
    c->wg[0] = 256; c->wg[1] = 1; c->wg[2] = 1;
    int s0 = add_stmt(c, 0, (int)dt, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "seed", MEM_GLOBAL, DIR_LOAD, dn, ds, ix_lin));
    add_stmt(c, 1, (int)dt, 1, 0, 0);
    add_stmt(c, 2, (int)dt, op == 0, op == 1, op == 2);
    add_stmt(c, 1, (int)dt, 1, 0, 0);
    int s4 = add_stmt(c, 0, (int)dt, 0, 0, 0);
    stmt_site(c, s4, add_site(c, "out", MEM_GLOBAL, DIR_STORE, dn, ds, ix_lin));
    c->walk = walk_fma;
    return 0;
}

/* local memory shuffle kernel.  P = {R, sync, G}.  Each work-item stores one
 * element into a 512-element local array, passes a barrier, then moves its
 * element between slot lid0 and slot 256+lid0 R/2 times (R local accesses in
 * the loop, 4 per iteration), optionally with a barrier per iteration, and
 * finally writes the element to global memory. */
static long long ix_lA(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)c; (void)g; (void)lv; return L0_;
}
static long long ix_lB(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)c; (void)g; (void)lv; return 256 + L0_;
}
static void walk_smem(ctx *c) {
    long long lv[1];
    X(c, 0, NULL);          /* v = in[gtid] ; s[lid0] = v */
    BAR(c);
    for (lv[0] = 0; lv[0] < c->P[0] / 4; lv[0]++) {
        X(c, 1, lv);        /* s[256+lid0] = s[lid0] */
        X(c, 2, lv);        /* s[lid0] = s[256+lid0] */
        if (c->P[1]) BAR(c);
    }
    X(c, 3, NULL);          /* out[gtid] = s[lid0] */
}
static void walk_smem2d(ctx *c) {
    long long lv[1];
    X(c, 0, NULL);
    BAR(c);
    for (lv[0] = 0; lv[0] < c->P[0] / 4; lv[0]++) {
        X(c, 1, lv);
        X(c, 2, lv);
    }
    X(c, 3, NULL);
}
static int setup_smem(ctx *c) {
    long long R = c->P[0], sync = c->P[1], G = c->P[2];
    if (R < 4 || R % 4 || sync < 0 || sync > 1 || G < 1) return -1;
    c->grid[0] = G; c->grid[1] = 1; c->grid[2] = 1;
    c->wg[0] = 256; c->wg[1] = 1; c->wg[2] = 1;
    int s0 = add_stmt(c, 0, DT_F32, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "in", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_lin));
    stmt_site(c, s0, add_site(c, "s_init", MEM_LOCAL, DIR_STORE, "float32", 4, ix_lA));
    int s1 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "s_ldA", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_lA));
    stmt_site(c, s1, add_site(c, "s_stB", MEM_LOCAL, DIR_STORE, "float32", 4, ix_lB));
    int s2 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s2, add_site(c, "s_ldB", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_lB));
    stmt_site(c, s2, add_site(c, "s_stA", MEM_LOCAL, DIR_STORE, "float32", 4, ix_lA));
    int s3 = add_stmt(c, 0, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "s_fin", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_lA));
    stmt_site(c, s3, add_site(c, "out", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_lin));
    c->walk = walk_smem;
    return 0;
}

/* 2-D local memory shuffle kernel (local accesses with a lid(1) stride, the
 * pattern of the stencil tiles' local memory).  P = {R, T, G}.  T x T
 * work-groups, local index a = T lid1 + lid0: each work-item stores its
 * element at slot a, passes a barrier, moves it between slots a and T^2 + a
 * R/2 times (R local accesses in the loop), and writes it to global memory
 * at G0-major offset T^2 gid0 + a. */
static long long ix_l2A(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return c->P[1] * L1_ + L0_;
}
static long long ix_l2B(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; long long T = c->P[1]; return T * T + T * L1_ + L0_;
}
static long long ix_l2g(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; long long T = c->P[1]; return T * T * G0 + T * L1_ + L0_;
}
static int setup_smem2d(ctx *c) {
    long long R = c->P[0], T = c->P[1], G = c->P[2];
    if (R < 4 || R % 4 || (T != 16 && T != 18) || G < 1) return -1;
    c->grid[0] = G; c->grid[1] = 1; c->grid[2] = 1;
    c->wg[0] = T; c->wg[1] = T; c->wg[2] = 1;
    int s0 = add_stmt(c, 0, DT_F32, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "in", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_l2g));
    stmt_site(c, s0, add_site(c, "s_init", MEM_LOCAL, DIR_STORE, "float32", 4, ix_l2A));
    int s1 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "s_ldA", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_l2A));
    stmt_site(c, s1, add_site(c, "s_stB", MEM_LOCAL, DIR_STORE, "float32", 4, ix_l2B));
    int s2 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s2, add_site(c, "s_ldB", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_l2B));
    stmt_site(c, s2, add_site(c, "s_stA", MEM_LOCAL, DIR_STORE, "float32", 4, ix_l2A));
    int s3 = add_stmt(c, 0, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "s_fin", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_l2A));
    stmt_site(c, s3, add_site(c, "out", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_l2g));
    c->walk = walk_smem2d;
    return 0;
}

/* local barrier kernel.  P = {B, G}: v = in[gtid]; B barriers; out[gtid] = v. */
static void walk_barrier(ctx *c) {
    X(c, 0, NULL);
    for (long long b = 0; b < c->P[0]; b++) BAR(c);
    X(c, 1, NULL);
}
static int setup_barrier(ctx *c) {
    long long B = c->P[0], G = c->P[1];
    if (B < 0 || G < 1) return -1;
    c->grid[0] = G; c->grid[1] = 1; c->grid[2] = 1;
    c->wg[0] = 256; c->wg[1] = 1; c->wg[2] = 1;
    int s0 = add_stmt(c, 0, DT_F32, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "in", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_lin));
    int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "out", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_lin));
    c->walk = walk_barrier;
    return 0;
}

/* local/global overlap kernel (Section "Modeling Operation Overlap"):
 * one global load, m local store-load pairs, one global store.  P = {m, N}. */
static void walk_overlap(ctx *c) {
    long long lv[1];
    X(c, 0, NULL);
    for (lv[0] = 0; lv[0] < c->P[0]; lv[0]++) { X(c, 1, lv); X(c, 2, lv); }
    X(c, 3, NULL);
}
static int setup_overlap(ctx *c) {
    long long m = c->P[0], N = c->P[1];
    if (m < 0 || N < 256 || N % 256) return -1;
    c->grid[0] = N / 256; c->grid[1] = 1; c->grid[2] = 1;
    c->wg[0] = 256; c->wg[1] = 1; c->wg[2] = 1;
    int s0 = add_stmt(c, 0, DT_F32, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "in", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_lin));
    int s1 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "s_st", MEM_LOCAL, DIR_STORE, "float32", 4, ix_lA));
    int s2 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s2, add_site(c, "s_ld", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_lA));
    int s3 = add_stmt(c, 0, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "out", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_lin));
    c->walk = walk_overlap;
    return 0;
}

/* empty kernel: G work-groups of 256 with no instructions.  P = {G}. */
static void walk_empty(ctx *c) { (void)c; }
static int setup_empty(ctx *c) {
    if (c->P[0] < 1) return -1;
    c->grid[0] = c->P[0]; c->grid[1] = 1; c->grid[2] = 1;
    c->wg[0] = 256; c->wg[1] = 1; c->wg[2] = 1;
    c->walk = walk_empty;
    return 0;
}

/* ======================================================================
 * Matrix multiplication (Sections "Illustrative Example", "Matrix
 * Multiplication"), C = A B, n x n fp32 row-major, 16x16 work-groups,
 * gid0 -> column tile, gid1 -> row tile.  P = {n}.
 * ====================================================================== */
static long long ix_mm_a_pf(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long n = c->P[0]; return n * (16 * G1 + L1_) + 16 * lv[0] + L0_;
}
static long long ix_mm_b_pf(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long n = c->P[0]; return n * (16 * lv[0] + L1_) + 16 * G0 + L0_;
}
static long long ix_mm_tile_st(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)c; (void)g; (void)lv; return 16 * L1_ + L0_;
}
static long long ix_mm_af_ld(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)c; (void)g; return 16 * L1_ + lv[1];
}
static long long ix_mm_bf_ld(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)c; (void)g; return 16 * lv[1] + L0_;
}
static long long ix_mm_c(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; long long n = c->P[0]; return n * (16 * G1 + L1_) + 16 * G0 + L0_;
}
static long long ix_mm_a_np(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long n = c->P[0]; return n * (16 * G1 + L1_) + lv[0];
}
static long long ix_mm_b_np(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long n = c->P[0]; return n * lv[0] + 16 * G0 + L0_;
}

/* variants: 0 PF, 1 noPF, 2 PF-a twin, 3 PF-b twin, 4 noPF-a twin, 5 noPF-b twin */
static void walk_mm(ctx *c) {
    long long n = c->P[0], v = c->D[0], lv[2];
    switch (v) {
    case 0:
        for (lv[0] = 0; lv[0] < n / 16; lv[0]++) {
            BAR(c);
            X(c, 0, lv);                      /* a tile -> local */
            X(c, 1, lv);                      /* b tile -> local */
            BAR(c);
            for (lv[1] = 0; lv[1] < 16; lv[1]++) X(c, 2, lv);   /* acc += af*bf */
        }
        X(c, 3, NULL);
        break;
    case 1:
        for (lv[0] = 0; lv[0] < n; lv[0]++) X(c, 0, lv);        /* acc += a*b */
        X(c, 1, NULL);
        break;
    case 2: case 3:
        for (lv[0] = 0; lv[0] < n / 16; lv[0]++) X(c, 0, lv);   /* tgt += a|b */
        X(c, 1, NULL);
        break;
    case 4: case 5:
        for (lv[0] = 0; lv[0] < n; lv[0]++) X(c, 0, lv);
        X(c, 1, NULL);
        break;
    }
}
static int setup_mm(ctx *c, int v) {
    long long n = c->P[0];
    if (n < 16 || n % 16) return -1;
    c->D[0] = v;
    c->grid[0] = n / 16; c->grid[1] = n / 16; c->grid[2] = 1;
    c->wg[0] = 16; c->wg[1] = 16; c->wg[2] = 1;
    if (v == 0) {
        int s0 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, "mm-PF-a", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_mm_a_pf));
        stmt_site(c, s0, add_site(c, "a_fetch_st", MEM_LOCAL, DIR_STORE, "float32", 4, ix_mm_tile_st));
        int s1 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "mm-PF-b", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_mm_b_pf));
        stmt_site(c, s1, add_site(c, "b_fetch_st", MEM_LOCAL, DIR_STORE, "float32", 4, ix_mm_tile_st));
        int s2 = add_stmt(c, 2, DT_F32, 0, 0, 1);
        stmt_site(c, s2, add_site(c, "a_fetch_ld", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_mm_af_ld));
        stmt_site(c, s2, add_site(c, "b_fetch_ld", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_mm_bf_ld));
        int s3 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s3, add_site(c, "c", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_mm_c));
    } else if (v == 1) {
        int s0 = add_stmt(c, 1, DT_F32, 0, 0, 1);
        stmt_site(c, s0, add_site(c, "mm-noPF-a", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_mm_a_np));
        stmt_site(c, s0, add_site(c, "mm-noPF-b", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_mm_b_np));
        int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "c", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_mm_c));
    } else {
        idx_fn f = v == 2 ? ix_mm_a_pf : v == 3 ? ix_mm_b_pf : v == 4 ? ix_mm_a_np : ix_mm_b_np;
        const char *tag = v == 2 ? "mm-PF-a" : v == 3 ? "mm-PF-b" : v == 4 ? "mm-noPF-a" : "mm-noPF-b";
        int s0 = add_stmt(c, 1, DT_F32, 1, 0, 0);
        stmt_site(c, s0, add_site(c, tag, MEM_GLOBAL, DIR_LOAD, "float32", 4, f));
        int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_mm_c));
    }
    c->walk = walk_mm;
    return 0;
}

/* ======================================================================
 * DG differentiation (Section "DG"): res[m,k,i] = sum_j D[m,i,j] u[k,j],
 * m < 3, D: 3 x Np x Np, u: Nel x Np, res: 3 x Nel x Np, all row-major fp32.
 * k = L0*gid0 + lid0 (k split by lsize0), i = L1*gid1 + lid1 (i split by
 * lsize1), guard i < Np.  P = {Np, Nel, L0, L1}.
 * variants: 0 noPF, 1 dmPF (D tiles L1 x L0 prefetched to local memory,
 * j split by L0), 2 noPF-u twin, 3 noPF-dm twin, 4 dmPF-u twin,
 * 5 dmPF-dm twin, 6 res twin (store pattern only), 7 uPF (L0 == L1; j
 * split by L1; per j tile the L0 x L1 tile of u is fetched to local memory,
 * work-item (lid0, lid1) fetching u[k = L0 gid0 + lid1, j = L1 jo + lid0];
 * loops j tile, j, m with three accumulators; the local value is read once
 * per j), 8 dmPF-T (dmPF on the transposed layouts uT[j, k] and
 * resT[m, i, k]), 9 uPF-u twin, 10 dmPF-T-u twin, 11 dmPF-T-res twin.
 * Twins without a kept store write tgt to tgt_dest[(L1 gid1 + lid1) * Nel + k]
 * (one entry per work-item, every work-item).
 * ====================================================================== */
#define DG_K(c, g, l) ((c)->P[2] * (g)[0] + (l)[0])
#define DG_I(c, g, l) ((c)->P[3] * (g)[1] + (l)[1])
static long long ix_dg_D(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0]; return Np * Np * lv[0] + Np * DG_I(c, g, l) + lv[1];
}
static long long ix_dg_u(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0]; return Np * DG_K(c, g, l) + lv[1];
}
static long long ix_dg_res(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0], Nel = c->P[1]; return Nel * Np * lv[0] + Np * DG_K(c, g, l) + DG_I(c, g, l);
}
/* dmPF: lv = {m, jo, ji} */
static long long ix_dg_Dfetch(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0], L0 = c->P[2];
    return Np * Np * lv[0] + Np * DG_I(c, g, l) + L0 * lv[1] + l[0];
}
static long long ix_dg_Dt_st(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return c->P[2] * l[1] + l[0];
}
static long long ix_dg_Dt_ld(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return c->P[2] * l[1] + lv[2];
}
static long long ix_dg_u_pf(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0], L0 = c->P[2]; return Np * DG_K(c, g, l) + L0 * lv[1] + lv[2];
}
static long long ix_dg_dest(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; return c->P[1] * DG_I(c, g, l) + DG_K(c, g, l);
}
/* uPF: lv = {jo, ji, m}; local tile uf[k_in][j_in] with row pitch L1 + 1 */
static long long ix_dg_upf_fetch(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0], L0 = c->P[2], L1 = c->P[3];
    return Np * (L0 * g[0] + l[1]) + L1 * lv[0] + l[0];
}
static long long ix_dg_uf_st(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return (c->P[3] + 1) * l[1] + l[0];
}
static long long ix_dg_uf_ld(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return (c->P[3] + 1) * l[0] + lv[1];
}
static long long ix_dg_upf_D(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0], L1 = c->P[3];
    return Np * Np * lv[2] + Np * DG_I(c, g, l) + L1 * lv[0] + lv[1];
}
/* dmPF-T: lv = {m, jo, ji}; uT[j, k] = Nel j + k, resT[m, i, k] = Nel Np m + Nel i + k */
static long long ix_dg_uT_pf(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Nel = c->P[1], L0 = c->P[2]; return Nel * (L0 * lv[1] + lv[2]) + DG_K(c, g, l);
}
static long long ix_dg_resT(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0], Nel = c->P[1]; return Nel * Np * lv[0] + Nel * DG_I(c, g, l) + DG_K(c, g, l);
}
static void walk_dg(ctx *c) {
    long long Np = c->P[0], L0 = c->P[2], v = c->D[0], lv[3];
    long long i = DG_I(c, c->g, c->l);
    long long nj = cdiv(Np, L0);
    switch (v) {
    case 0: case 2: case 3:
        if (i < Np)
            for (lv[0] = 0; lv[0] < 3; lv[0]++) {
                for (lv[1] = 0; lv[1] < Np; lv[1]++) X(c, 0, lv);
                if (v == 0) X(c, 1, lv);
            }
        if (v != 0) X(c, 1, NULL);
        break;
    case 1:
        for (lv[0] = 0; lv[0] < 3; lv[0]++) {
            for (lv[1] = 0; lv[1] < nj; lv[1]++) {
                BAR(c);
                if (i < Np && L0 * lv[1] + c->l[0] < Np) X(c, 0, lv);
                BAR(c);
                if (i < Np)
                    for (lv[2] = 0; lv[2] < L0; lv[2]++)
                        if (L0 * lv[1] + lv[2] < Np) X(c, 1, lv);
            }
            if (i < Np) X(c, 2, lv);
        }
        break;
    case 4:
        if (i < Np)
            for (lv[0] = 0; lv[0] < 3; lv[0]++)
                for (lv[1] = 0; lv[1] < nj; lv[1]++)
                    for (lv[2] = 0; lv[2] < L0; lv[2]++)
                        if (L0 * lv[1] + lv[2] < Np) X(c, 0, lv);
        X(c, 1, NULL);
        break;
    case 5:
        for (lv[0] = 0; lv[0] < 3; lv[0]++)
            for (lv[1] = 0; lv[1] < nj; lv[1]++)
                if (i < Np && L0 * lv[1] + c->l[0] < Np) X(c, 0, lv);
        X(c, 1, NULL);
        break;
    case 6: case 11:
        if (i < Np)
            for (lv[0] = 0; lv[0] < 3; lv[0]++) X(c, 0, lv);
        break;
    case 7: {
        long long L1 = c->P[3], njl = cdiv(Np, L1);
        for (lv[0] = 0; lv[0] < njl; lv[0]++) {
            BAR(c);
            if (L1 * lv[0] + c->l[0] < Np) X(c, 0, lv);
            BAR(c);
            if (i < Np)
                for (lv[1] = 0; lv[1] < L1 && L1 * lv[0] + lv[1] < Np; lv[1]++) {
                    X(c, 1, lv);
                    for (lv[2] = 0; lv[2] < 3; lv[2]++) X(c, 2, lv);
                }
        }
        if (i < Np)
            for (lv[0] = 0; lv[0] < 3; lv[0]++) X(c, 3, lv);
        break; }
    case 8:
        for (lv[0] = 0; lv[0] < 3; lv[0]++) {
            for (lv[1] = 0; lv[1] < nj; lv[1]++) {
                BAR(c);
                if (i < Np && L0 * lv[1] + c->l[0] < Np) X(c, 0, lv);
                BAR(c);
                if (i < Np)
                    for (lv[2] = 0; lv[2] < L0; lv[2]++)
                        if (L0 * lv[1] + lv[2] < Np) X(c, 1, lv);
            }
            if (i < Np) X(c, 2, lv);
        }
        break;
    case 9: {
        long long L1 = c->P[3], njl = cdiv(Np, L1);
        for (lv[0] = 0; lv[0] < njl; lv[0]++)
            if (L1 * lv[0] + c->l[0] < Np) X(c, 0, lv);
        X(c, 1, NULL);
        break; }
    case 10:
        if (i < Np)
            for (lv[0] = 0; lv[0] < 3; lv[0]++)
                for (lv[1] = 0; lv[1] < nj; lv[1]++)
                    for (lv[2] = 0; lv[2] < L0; lv[2]++)
                        if (L0 * lv[1] + lv[2] < Np) X(c, 0, lv);
        X(c, 1, NULL);
        break;
    }
}
static int setup_dg(ctx *c, int v) {
    long long Np = c->P[0], Nel = c->P[1], L0 = c->P[2], L1 = c->P[3];
    if (Np < 1 || Nel < 1 || L0 < 1 || L1 < 1 || L0 * L1 > 1024 || Nel % L0) return -1;
    c->D[0] = v;
    c->grid[0] = Nel / L0; c->grid[1] = cdiv(Np, L1); c->grid[2] = 1;
    c->wg[0] = L0; c->wg[1] = L1; c->wg[2] = 1;
    char t_nu[48], t_ndm[48], t_pu[48], t_pdm[48], t_res[48];
    snprintf(t_nu, sizeof t_nu, "dg-noPF-u-%dx%d", (int)L0, (int)L1);
    snprintf(t_ndm, sizeof t_ndm, "dg-noPF-dm-%dx%d", (int)L0, (int)L1);
    snprintf(t_pu, sizeof t_pu, "dg-dmPF-u-%dx%d", (int)L0, (int)L1);
    snprintf(t_pdm, sizeof t_pdm, "dg-dmPF-dm-%dx%d", (int)L0, (int)L1);
    snprintf(t_res, sizeof t_res, "dg-res-%dx%d", (int)L0, (int)L1);
    char t_uu[48], t_tu[48], t_tres[48];
    snprintf(t_uu, sizeof t_uu, "dg-uPF-u-%dx%d", (int)L0, (int)L1);
    snprintf(t_tu, sizeof t_tu, "dg-dmPFT-u-%dx%d", (int)L0, (int)L1);
    snprintf(t_tres, sizeof t_tres, "dg-dmPFT-res-%dx%d", (int)L0, (int)L1);
    switch (v) {
    case 0: {
        int s0 = add_stmt(c, 2, DT_F32, 0, 0, 1);
        stmt_site(c, s0, add_site(c, t_ndm, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_D));
        stmt_site(c, s0, add_site(c, t_nu, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_u));
        int s1 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, t_res, MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_res));
        break; }
    case 1: {
        int s0 = add_stmt(c, 2, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, t_pdm, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_Dfetch));
        stmt_site(c, s0, add_site(c, "dm_fetch_st", MEM_LOCAL, DIR_STORE, "float32", 4, ix_dg_Dt_st));
        int s1 = add_stmt(c, 3, DT_F32, 0, 0, 1);
        stmt_site(c, s1, add_site(c, "dm_fetch_ld", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_dg_Dt_ld));
        stmt_site(c, s1, add_site(c, t_pu, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_u_pf));
        int s2 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s2, add_site(c, t_res, MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_res));
        break; }
    case 2: case 3: {
        int s0 = add_stmt(c, 2, DT_F32, 1, 0, 0);
        if (v == 2) stmt_site(c, s0, add_site(c, t_nu, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_u));
        else stmt_site(c, s0, add_site(c, t_ndm, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_D));
        int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_dest));
        break; }
    case 4: {
        int s0 = add_stmt(c, 3, DT_F32, 1, 0, 0);
        stmt_site(c, s0, add_site(c, t_pu, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_u_pf));
        int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_dest));
        break; }
    case 5: {
        int s0 = add_stmt(c, 2, DT_F32, 1, 0, 0);
        stmt_site(c, s0, add_site(c, t_pdm, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_Dfetch));
        int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_dest));
        break; }
    case 6: {
        int s0 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, t_res, MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_res));
        break; }
    case 7: {
        if (L0 != L1) return -1;
        int s0 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, t_uu, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_upf_fetch));
        stmt_site(c, s0, add_site(c, "u_fetch_st", MEM_LOCAL, DIR_STORE, "float32", 4, ix_dg_uf_st));
        int s1 = add_stmt(c, 2, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "u_fetch_ld", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_dg_uf_ld));
        int s2 = add_stmt(c, 3, DT_F32, 0, 0, 1);
        stmt_site(c, s2, add_site(c, t_ndm, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_upf_D));
        int s3 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s3, add_site(c, t_res, MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_res));
        break; }
    case 8: {
        int s0 = add_stmt(c, 2, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, t_pdm, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_Dfetch));
        stmt_site(c, s0, add_site(c, "dm_fetch_st", MEM_LOCAL, DIR_STORE, "float32", 4, ix_dg_Dt_st));
        int s1 = add_stmt(c, 3, DT_F32, 0, 0, 1);
        stmt_site(c, s1, add_site(c, "dm_fetch_ld", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_dg_Dt_ld));
        stmt_site(c, s1, add_site(c, t_tu, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_uT_pf));
        int s2 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s2, add_site(c, t_tres, MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_resT));
        break; }
    case 9: {
        if (L0 != L1) return -1;
        int s0 = add_stmt(c, 1, DT_F32, 1, 0, 0);
        stmt_site(c, s0, add_site(c, t_uu, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_upf_fetch));
        int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_dest));
        break; }
    case 10: {
        int s0 = add_stmt(c, 3, DT_F32, 1, 0, 0);
        stmt_site(c, s0, add_site(c, t_tu, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dg_uT_pf));
        int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_dest));
        break; }
    case 11: {
        int s0 = add_stmt(c, 1, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, t_tres, MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dg_resT));
        break; }
    default: return -1;
    }
    c->walk = walk_dg;
    return 0;
}

/* ======================================================================
 * 2-D five-point finite difference stencil (Section "Finite Differences"):
 * res[i,j] = c0*u[i+1,j+1] + c1*(u[i,j+1] + u[i+2,j+1] + u[i+1,j] + u[i+1,j+2]),
 * u: (n+2) x (n+2), res: n x n, fp32 row-major.  P = {n}.
 * variants: 0 tile (16x16 work-group fetches a 16x16 tile of u to local
 * memory, the 14x14 interior computes, group stride 14), 1 direct (16x16
 * work-group, one output per work-item, five global loads), 2 tile-u twin,
 * 3 tile-res twin, 4 direct-u twin, 5 direct-res twin, 6 tile18 (18x18
 * work-group fetches an 18x18 tile, the 16x16 interior computes, group
 * stride 16), 7 tile18-u twin, 8 tile18-res twin.
 * Twins without a kept store write to
 * tgt_dest[(T gid1 + lid1)*(T G0) + T gid0 + lid0], T the work-group width.
 * ====================================================================== */
#define FD_W(c) ((c)->P[0] + 2)
#define FD_T(c) ((c)->D[1])            /* tile (work-group) width: 16 or 18 */
static long long ix_fd_fetch(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; long long s = FD_T(c) - 2; return FD_W(c) * (s * G1 + L1_) + s * G0 + L0_;
}
static long long ix_fd_tile_st(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return FD_T(c) * L1_ + L0_;
}
static long long ix_fd_tC(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return FD_T(c) * L1_ + L0_;
}
static long long ix_fd_tN(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return FD_T(c) * (L1_ - 1) + L0_;
}
static long long ix_fd_tS(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return FD_T(c) * (L1_ + 1) + L0_;
}
static long long ix_fd_tW(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return FD_T(c) * L1_ + L0_ - 1;
}
static long long ix_fd_tE(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)lv; return FD_T(c) * L1_ + L0_ + 1;
}
static long long ix_fd_res_tile(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; long long s = FD_T(c) - 2; return c->P[0] * (s * G1 + L1_ - 1) + s * G0 + L0_ - 1;
}
#define FD_DI(c, g, l) (16 * (g)[1] + (l)[1])
#define FD_DJ(c, g, l) (16 * (g)[0] + (l)[0])
static long long ix_fd_uC(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; return FD_W(c) * (FD_DI(c, g, l) + 1) + FD_DJ(c, g, l) + 1;
}
static long long ix_fd_uN(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; return FD_W(c) * FD_DI(c, g, l) + FD_DJ(c, g, l) + 1;
}
static long long ix_fd_uS(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; return FD_W(c) * (FD_DI(c, g, l) + 2) + FD_DJ(c, g, l) + 1;
}
static long long ix_fd_uW(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; return FD_W(c) * (FD_DI(c, g, l) + 1) + FD_DJ(c, g, l);
}
static long long ix_fd_uE(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; return FD_W(c) * (FD_DI(c, g, l) + 1) + FD_DJ(c, g, l) + 2;
}
static long long ix_fd_res_direct(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; return c->P[0] * FD_DI(c, g, l) + FD_DJ(c, g, l);
}
static long long ix_fd_dest(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv; long long T = c->wg[0]; return T * c->grid[0] * (T * G1 + L1_) + T * G0 + L0_;
}
static void walk_fd(ctx *c) {
    long long n = c->P[0], W = n + 2, v = c->D[0];
    const long long *g = c->g, *l = c->l;
    if (v == 0 || v == 2 || v == 3 || v >= 6) {
        long long s = FD_T(c) - 2, r = s * G1 + L1_, q = s * G0 + L0_;
        int fetch = r < W && q < W;
        int comp = L0_ >= 1 && L0_ <= s && L1_ >= 1 && L1_ <= s && r - 1 < n && q - 1 < n;
        if (v == 0 || v == 6) {
            if (fetch) X(c, 0, NULL);
            BAR(c);
            if (comp) X(c, 1, NULL);
        } else if (v == 2 || v == 7) {
            if (fetch) X(c, 0, NULL);
            X(c, 1, NULL);
        } else {
            if (comp) X(c, 0, NULL);
        }
    } else {
        long long i = FD_DI(c, g, l), j = FD_DJ(c, g, l);
        int comp = i < n && j < n;
        if (v == 1 || v == 5) { if (comp) X(c, 0, NULL); }
        else {
            if (comp) for (int s = 0; s < 5; s++) X(c, s, NULL);
            X(c, 5, NULL);
        }
    }
}
static int setup_fd(ctx *c, int v) {
    long long n = c->P[0];
    if (n < 1) return -1;
    c->D[0] = v;
    c->D[1] = v >= 6 ? 18 : 16;
    c->wg[0] = c->D[1]; c->wg[1] = c->D[1]; c->wg[2] = 1;
    if (v == 0 || v == 2 || v == 3 || v >= 6) { c->grid[0] = cdiv(n, c->D[1] - 2); c->grid[1] = c->grid[0]; }
    else { c->grid[0] = cdiv(n, 16); c->grid[1] = cdiv(n, 16); }
    c->grid[2] = 1;
    const char *t_u = v >= 6 ? "fd-tile18-u" : "fd-tile-u", *t_res = v >= 6 ? "fd-tile18-res" : "fd-tile-res";
    switch (v) {
    case 0: case 6: {
        int s0 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, t_u, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_fd_fetch));
        stmt_site(c, s0, add_site(c, "u_fetch_st", MEM_LOCAL, DIR_STORE, "float32", 4, ix_fd_tile_st));
        int s1 = add_stmt(c, 0, DT_F32, 3, 1, 1);
        stmt_site(c, s1, add_site(c, "u_fetch_c", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_fd_tC));
        stmt_site(c, s1, add_site(c, "u_fetch_n", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_fd_tN));
        stmt_site(c, s1, add_site(c, "u_fetch_s", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_fd_tS));
        stmt_site(c, s1, add_site(c, "u_fetch_w", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_fd_tW));
        stmt_site(c, s1, add_site(c, "u_fetch_e", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_fd_tE));
        stmt_site(c, s1, add_site(c, t_res, MEM_GLOBAL, DIR_STORE, "float32", 4, ix_fd_res_tile));
        break; }
    case 1: {
        int s0 = add_stmt(c, 0, DT_F32, 3, 1, 1);
        stmt_site(c, s0, add_site(c, "u_c", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_fd_uC));
        stmt_site(c, s0, add_site(c, "u_n", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_fd_uN));
        stmt_site(c, s0, add_site(c, "u_s", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_fd_uS));
        stmt_site(c, s0, add_site(c, "u_w", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_fd_uW));
        stmt_site(c, s0, add_site(c, "u_e", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_fd_uE));
        stmt_site(c, s0, add_site(c, "res", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_fd_res_direct));
        break; }
    case 2: case 7: {
        int s0 = add_stmt(c, 0, DT_F32, 1, 0, 0);
        stmt_site(c, s0, add_site(c, t_u, MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_fd_fetch));
        int s1 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s1, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_fd_dest));
        break; }
    case 3: case 8: {
        int s0 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, t_res, MEM_GLOBAL, DIR_STORE, "float32", 4, ix_fd_res_tile));
        break; }
    case 4: {
        static const char *nm[5] = {"u_c", "u_n", "u_s", "u_w", "u_e"};
        idx_fn fs[5] = {ix_fd_uC, ix_fd_uN, ix_fd_uS, ix_fd_uW, ix_fd_uE};
        for (int s = 0; s < 5; s++) {
            int st = add_stmt(c, 0, DT_F32, 1, 0, 0);
            stmt_site(c, st, add_site(c, nm[s], MEM_GLOBAL, DIR_LOAD, "float32", 4, fs[s]));
        }
        int s5 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s5, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_fd_dest));
        break; }
    case 5: {
        int s0 = add_stmt(c, 0, DT_F32, 0, 0, 0);
        stmt_site(c, s0, add_site(c, "res", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_fd_res_direct));
        break; }
    default: return -1;
    }
    c->walk = walk_fd;
    return 0;
}

/* ======================================================================
 * Register-tiled SIMT matmul family (autotuning space): C = A B, n x n fp32,
 * 16-byte vector (float32x4) global accesses.  P = {n, BM, BN, BK}.
 * Work-group L0 x L1 = (BN/8) x (BM/8); each work-item owns an 8 x 8 block
 * of C (rows 8 lid1 .., vector columns lid0 and L0 + lid0).  Per k tile
 * (BK wide):
 *   barrier;
 *   A tile: rows lid1 + L1 r (r < 8), vector columns c = lid0 + L0 q
 *           (q < ceil(KC/L0), guard c < KC, KC = BK/4); stored transposed as
 *           four scalars As[(4c + j) (BM + 4) + row] (j < 4; rows padded by 4
 *           so that the 8 columns of a warp fall on 4 banks, not 1);
 *   B tile: rows lid1 + L1 r (r < ceil(BK/L1), guard row < BK), vector
 *           columns c = lid0 + L0 q (q < 2); stored as one vector Bs[row NC + c];
 *   barrier;
 *   kk < BK: two vector loads of As (8 values at kk (BM + 4) + 8 lid1), two of Bs
 *           (vectors lid0 and L0 + lid0 of row kk), 64 multiply-adds.
 * Finally 8 x 2 vector stores of C (rows 8 lid1 + i, vector columns
 * NC gid0 + lid0 + L0 j).  Requires n divisible by BM, BN, BK.
 * Index units: float32x4 (vectors) for global and Bs / As vector loads,
 * float32 for the scalar As stores.
 * ====================================================================== */
#define SM_N(c) ((c)->P[0])
#define SM_BM(c) ((c)->P[1])
#define SM_BN(c) ((c)->P[2])
#define SM_BK(c) ((c)->P[3])
static long long ix_sm_a(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    /* lv = {kt, r, q} */
    long long n4 = SM_N(c) / 4, KC = SM_BK(c) / 4, L0 = SM_BN(c) / 8, L1 = SM_BM(c) / 8;
    return n4 * (SM_BM(c) * G1 + L1_ + L1 * lv[1]) + KC * lv[0] + L0_ + L0 * lv[2];
}
static long long ix_sm_ast(const ctx *c, const long long *g, const long long *l, const long long *lv, int j) {
    (void)g;
    long long L0 = SM_BN(c) / 8, L1 = SM_BM(c) / 8, BMP = SM_BM(c) + 4;
    return (4 * (L0_ + L0 * lv[2]) + j) * BMP + L1_ + L1 * lv[1];
}
static long long ix_sm_ast0(const ctx *c, const long long *g, const long long *l, const long long *lv) { return ix_sm_ast(c, g, l, lv, 0); }
static long long ix_sm_ast1(const ctx *c, const long long *g, const long long *l, const long long *lv) { return ix_sm_ast(c, g, l, lv, 1); }
static long long ix_sm_ast2(const ctx *c, const long long *g, const long long *l, const long long *lv) { return ix_sm_ast(c, g, l, lv, 2); }
static long long ix_sm_ast3(const ctx *c, const long long *g, const long long *l, const long long *lv) { return ix_sm_ast(c, g, l, lv, 3); }
static long long ix_sm_b(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long n4 = SM_N(c) / 4, L0 = SM_BN(c) / 8, L1 = SM_BM(c) / 8, NC = SM_BN(c) / 4;
    return n4 * (SM_BK(c) * lv[0] + L1_ + L1 * lv[1]) + NC * G0 + L0_ + L0 * lv[2];
}
static long long ix_sm_bst(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g;
    long long L0 = SM_BN(c) / 8, L1 = SM_BM(c) / 8, NC = SM_BN(c) / 4;
    return (L1_ + L1 * lv[1]) * NC + L0_ + L0 * lv[2];
}
static long long ix_sm_ald(const ctx *c, const long long *g, const long long *l, const long long *lv, int h) {
    (void)g; return lv[1] * ((SM_BM(c) + 4) / 4) + 2 * L1_ + h;
}
static long long ix_sm_ald0(const ctx *c, const long long *g, const long long *l, const long long *lv) { return ix_sm_ald(c, g, l, lv, 0); }
static long long ix_sm_ald1(const ctx *c, const long long *g, const long long *l, const long long *lv) { return ix_sm_ald(c, g, l, lv, 1); }
static long long ix_sm_bld(const ctx *c, const long long *g, const long long *l, const long long *lv, int h) {
    (void)g; return lv[1] * (SM_BN(c) / 4) + L0_ + (SM_BN(c) / 8) * h;
}
static long long ix_sm_bld0(const ctx *c, const long long *g, const long long *l, const long long *lv) { return ix_sm_bld(c, g, l, lv, 0); }
static long long ix_sm_bld1(const ctx *c, const long long *g, const long long *l, const long long *lv) { return ix_sm_bld(c, g, l, lv, 1); }
static long long ix_sm_c(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    /* lv = {i, j} */
    long long n4 = SM_N(c) / 4, NC = SM_BN(c) / 4;
    return n4 * (SM_BM(c) * G1 + 8 * L1_ + lv[0]) + NC * G0 + L0_ + (SM_BN(c) / 8) * lv[1];
}
static void walk_simt(ctx *c) {
    long long n = SM_N(c), BK = SM_BK(c), KC = BK / 4, L0 = SM_BN(c) / 8, L1 = SM_BM(c) / 8;
    long long lv[3];
    long long qa = cdiv(KC, L0), rb = cdiv(BK, L1);
    for (lv[0] = 0; lv[0] < n / BK; lv[0]++) {
        BAR(c);
        for (lv[1] = 0; lv[1] < 8; lv[1]++)
            for (lv[2] = 0; lv[2] < qa; lv[2]++)
                if (c->l[0] + L0 * lv[2] < KC) X(c, 0, lv);
        for (lv[1] = 0; lv[1] < rb; lv[1]++)
            for (lv[2] = 0; lv[2] < 2; lv[2]++)
                if (c->l[1] + L1 * lv[1] < BK) X(c, 1, lv);
        BAR(c);
        long long kk[2];
        kk[0] = lv[0];
        for (kk[1] = 0; kk[1] < BK; kk[1]++) X(c, 2, kk);
    }
    for (lv[0] = 0; lv[0] < 8; lv[0]++)
        for (lv[1] = 0; lv[1] < 2; lv[1]++) X(c, 3, lv);
}
static int setup_simt(ctx *c) {
    long long n = SM_N(c), BM = SM_BM(c), BN = SM_BN(c), BK = SM_BK(c);
    if (BM < 8 || BN < 8 || BK < 4 || BM % 8 || BN % 8 || BK % 4 || n % BM || n % BN || n % BK || n % 4) return -1;
    if ((BM / 8) * (BN / 8) > 1024) return -1;
    c->grid[0] = n / BN; c->grid[1] = n / BM; c->grid[2] = 1;
    c->wg[0] = BN / 8; c->wg[1] = BM / 8; c->wg[2] = 1;
    int s0 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "simt-a", MEM_GLOBAL, DIR_LOAD, "float32x4", 16, ix_sm_a));
    stmt_site(c, s0, add_site(c, "As_st0", MEM_LOCAL, DIR_STORE, "float32", 4, ix_sm_ast0));
    stmt_site(c, s0, add_site(c, "As_st1", MEM_LOCAL, DIR_STORE, "float32", 4, ix_sm_ast1));
    stmt_site(c, s0, add_site(c, "As_st2", MEM_LOCAL, DIR_STORE, "float32", 4, ix_sm_ast2));
    stmt_site(c, s0, add_site(c, "As_st3", MEM_LOCAL, DIR_STORE, "float32", 4, ix_sm_ast3));
    int s1 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "simt-b", MEM_GLOBAL, DIR_LOAD, "float32x4", 16, ix_sm_b));
    stmt_site(c, s1, add_site(c, "Bs_st", MEM_LOCAL, DIR_STORE, "float32x4", 16, ix_sm_bst));
    int s2 = add_stmt(c, 2, DT_F32, 0, 0, 64);
    stmt_site(c, s2, add_site(c, "As_ld0", MEM_LOCAL, DIR_LOAD, "float32x4", 16, ix_sm_ald0));
    stmt_site(c, s2, add_site(c, "As_ld1", MEM_LOCAL, DIR_LOAD, "float32x4", 16, ix_sm_ald1));
    stmt_site(c, s2, add_site(c, "Bs_ld0", MEM_LOCAL, DIR_LOAD, "float32x4", 16, ix_sm_bld0));
    stmt_site(c, s2, add_site(c, "Bs_ld1", MEM_LOCAL, DIR_LOAD, "float32x4", 16, ix_sm_bld1));
    int s3 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "simt-c", MEM_GLOBAL, DIR_STORE, "float32x4", 16, ix_sm_c));
    c->walk = walk_simt;
    return 0;
}

/* ======================================================================
 * BF16 tensor-core matmul: C = A Bt^T, A and Bt n x n bf16 row-major, C fp32.
 * P = {n}.  Work-group of 128 work-items (1-D), grid (n/256, n/128), one
 * 128 x 256 tile of C per work-group.  Work-item 0 copies, per 64-wide k
 * tile, the 128 x 64 box of A and the 256 x 64 box of Bt (described element
 * by element); work-item 32 issues four 128 x 256 x 16 multiply-add
 * instructions per k tile; every work-item stores its C row as 8 x 8
 * float32x4 vectors; three barriers.
 * ====================================================================== */
static long long ix_tc_a(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)l; long long n = c->P[0]; return n * (128 * G1 + lv[1]) + 64 * lv[0] + lv[2];
}
static long long ix_tc_b(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)l; long long n = c->P[0]; return n * (256 * G0 + lv[1]) + 64 * lv[0] + lv[2];
}
static long long ix_tc_c(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long n = c->P[0]; return (n / 4) * (128 * G1 + L0_) + 64 * G0 + 8 * lv[0] + lv[1];
}
static void walk_tc(ctx *c) {
    long long n = c->P[0], lv[3];
    BAR(c);
    if (c->l[0] == 0)
        for (lv[0] = 0; lv[0] < n / 64; lv[0]++) {
            for (lv[1] = 0; lv[1] < 128; lv[1]++)
                for (lv[2] = 0; lv[2] < 64; lv[2]++) X(c, 0, lv);
            for (lv[1] = 0; lv[1] < 256; lv[1]++)
                for (lv[2] = 0; lv[2] < 64; lv[2]++) X(c, 1, lv);
        }
    if (c->l[0] == 32)
        for (lv[0] = 0; lv[0] < n / 64; lv[0]++)
            for (lv[1] = 0; lv[1] < 4; lv[1]++) X(c, 2, lv);
    for (lv[0] = 0; lv[0] < 8; lv[0]++)
        for (lv[1] = 0; lv[1] < 8; lv[1]++) X(c, 3, lv);
    BAR(c);
    BAR(c);
}
static int setup_tc(ctx *c) {
    long long n = c->P[0];
    if (n < 256 || n % 256) return -1;
    c->grid[0] = n / 256; c->grid[1] = n / 128; c->grid[2] = 1;
    c->wg[0] = 128; c->wg[1] = 1; c->wg[2] = 1;
    int s0 = add_stmt(c, 3, DT_BF16, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "tc-a", MEM_GLOBAL, DIR_LOAD, "bfloat16", 2, ix_tc_a));
    int s1 = add_stmt(c, 3, DT_BF16, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "tc-b", MEM_GLOBAL, DIR_LOAD, "bfloat16", 2, ix_tc_b));
    add_stmt(c, 2, DT_BF16, 0, 0, 128 * 256 * 16);
    int s3 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "tc-c", MEM_GLOBAL, DIR_STORE, "float32x4", 16, ix_tc_c));
    c->walk = walk_tc;
    return 0;
}

/* 256 x 256 tile variant: a 256-work-item group per tile; work-item 0
 * copies a 256x64 box of A and a 256x64 box of Bt per 64-wide k tile,
 * work-item 32 issues eight 128x256x16 multiply-adds per k tile (two row
 * halves sharing the Bt box), work-item t stores row t of the tile (64
 * 16-byte vectors); three barriers. */
static long long ix_tcw_a(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)l; long long n = c->P[0]; return n * (256 * G1 + lv[1]) + 64 * lv[0] + lv[2];
}
static long long ix_tcw_c(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long n = c->P[0]; return (n / 4) * (256 * G1 + L0_) + 64 * G0 + 8 * lv[0] + lv[1];
}
static void walk_tcw(ctx *c) {
    long long n = c->P[0], lv[3];
    BAR(c);
    if (c->l[0] == 0)
        for (lv[0] = 0; lv[0] < n / 64; lv[0]++) {
            for (lv[1] = 0; lv[1] < 256; lv[1]++)
                for (lv[2] = 0; lv[2] < 64; lv[2]++) X(c, 0, lv);
            for (lv[1] = 0; lv[1] < 256; lv[1]++)
                for (lv[2] = 0; lv[2] < 64; lv[2]++) X(c, 1, lv);
        }
    if (c->l[0] == 32)
        for (lv[0] = 0; lv[0] < n / 64; lv[0]++)
            for (lv[1] = 0; lv[1] < 8; lv[1]++) X(c, 2, lv);
    for (lv[0] = 0; lv[0] < 8; lv[0]++)
        for (lv[1] = 0; lv[1] < 8; lv[1]++) X(c, 3, lv);
    BAR(c);
    BAR(c);
}
static int setup_tcw(ctx *c) {
    long long n = c->P[0];
    if (n < 256 || n % 256) return -1;
    c->grid[0] = n / 256; c->grid[1] = n / 256; c->grid[2] = 1;
    c->wg[0] = 256; c->wg[1] = 1; c->wg[2] = 1;
    int s0 = add_stmt(c, 3, DT_BF16, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "tc-a", MEM_GLOBAL, DIR_LOAD, "bfloat16", 2, ix_tcw_a));
    int s1 = add_stmt(c, 3, DT_BF16, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "tc-b", MEM_GLOBAL, DIR_LOAD, "bfloat16", 2, ix_tc_b));
    add_stmt(c, 2, DT_BF16, 0, 0, 128 * 256 * 16);
    int s3 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "tc-c", MEM_GLOBAL, DIR_STORE, "float32x4", 16, ix_tcw_c));
    c->walk = walk_tcw;
    return 0;
}

/* FP64 reference of C = A Bt^T over bf16 inputs (uint16 bit patterns) */
static double bf16_value(unsigned short h) {
    union { unsigned int u; float f; } v;
    v.u = (unsigned int)h << 16;
    return (double)v.f;
}
void oracle_mm_tc_ref(long long m, long long n, long long k, const unsigned short *a, const unsigned short *bt,
                      double *c, double *cabs) {
    /* a: m x k, bt: n x k, c: m x n */
    for (long long i = 0; i < m; i++)
        for (long long j = 0; j < n; j++) {
            double s = 0.0, sa = 0.0;
            for (long long q = 0; q < k; q++) {
                double p = bf16_value(a[k * i + q]) * bf16_value(bt[k * j + q]);
                s += p; sa += fabs(p);
            }
            c[n * i + j] = s; cabs[n * i + j] = sa;
        }
}

/* ======================================================================
 * Stencil tile family (TMA-staged): P = {n, BX, BY, V}; input rows of pitch
 * n + 4; work-group (BX/V) x BY, grid (n/BX, n/BY).  Work-item (0,0) copies
 * the (BY+2) x (BX+4) box at (row BY gid1, column BX gid0) element by
 * element; one barrier; every work-item then loads its V + 2 centre-row
 * values (columns V lid0 + q, q = 0..V+1), and for q = 1..V its north and
 * south values with one output each (3 add + 1 mul + 1 madd), and stores its
 * V outputs as V/4 float32x4 vectors.
 * ====================================================================== */
#define FB_BX(c) ((c)->P[1])
#define FB_BY(c) ((c)->P[2])
#define FB_V(c) ((c)->P[3])
static long long ix_fb_u(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)l; long long P = c->P[0] + 4; return P * (FB_BY(c) * G1 + lv[0]) + FB_BX(c) * G0 + lv[1];
}
static long long fb_t(const ctx *c, const long long *l, long long row, long long col) {
    return (FB_BX(c) + 4) * (L1_ + row) + FB_V(c) * L0_ + col;
}
static long long ix_fb_c(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return fb_t(c, l, 1, lv[0]);
}
static long long ix_fb_n(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return fb_t(c, l, 0, lv[0]);
}
static long long ix_fb_s(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return fb_t(c, l, 2, lv[0]);
}
static long long ix_fb_res(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long n = c->P[0];
    return (n / 4) * (FB_BY(c) * G1 + L1_) + (FB_BX(c) / 4) * G0 + (FB_V(c) / 4) * L0_ + lv[0];
}
static void walk_fdb(ctx *c) {
    long long lv[2];
    if (c->l[0] == 0 && c->l[1] == 0)
        for (lv[0] = 0; lv[0] < FB_BY(c) + 2; lv[0]++)
            for (lv[1] = 0; lv[1] < FB_BX(c) + 4; lv[1]++) X(c, 0, lv);
    BAR(c);
    for (lv[0] = 0; lv[0] < FB_V(c) + 2; lv[0]++) X(c, 1, lv);
    for (lv[0] = 1; lv[0] <= FB_V(c); lv[0]++) X(c, 2, lv);
    for (lv[0] = 0; lv[0] < FB_V(c) / 4; lv[0]++) X(c, 3, lv);
}
static int setup_fdb(ctx *c) {
    long long n = c->P[0], BX = c->P[1], BY = c->P[2], V = c->P[3];
    if ((V != 4 && V != 8) || BX < V || BX % V || BY < 1 || n % BX || n % BY || n % 4) return -1;
    c->grid[0] = n / BX; c->grid[1] = n / BY; c->grid[2] = 1;
    c->wg[0] = BX / V; c->wg[1] = BY; c->wg[2] = 1;
    int s0 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "fdb-u", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_fb_u));
    int s1 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "t_c", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_fb_c));
    int s2 = add_stmt(c, 1, DT_F32, 3, 1, 1);
    stmt_site(c, s2, add_site(c, "t_n", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_fb_n));
    stmt_site(c, s2, add_site(c, "t_s", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_fb_s));
    int s3 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "fdb-res", MEM_GLOBAL, DIR_STORE, "float32x4", 16, ix_fb_res));
    c->walk = walk_fdb;
    return 0;
}

/* ======================================================================
 * DG tile (GB300 form of the DG derivative): P = {Np, Nel}.  For one m
 * (gid0 < 3) and 128 elements (gid1): res[m, k, i] = sum_j D[m, i, j]
 * u[k, j] as one matrix product.  NB = ceil(Np / 16) columns per
 * work-item, XL = ceil(Np / NB) x-lanes: work-group XL x 16, grid
 * (3, ceil(Nel / 128)); node rows i padded to NPP = XL NB with zeros, j in
 * Q = ceil(Np / 2) pairs (8-byte vectors), zero beyond Np; Dt row pitch PD
 * floats (PD >= 2 Q, PD % 32 == 2).
 *  - D staging: for row block ib < ceil(NPP / 16) and pair block
 *    qb < ceil(Q / XL): work-item (lid0, lid1) handles i = lid1 + 16 ib and
 *    q = lid0 + XL qb; for q < Q and i < NPP: when i < Np it loads
 *    D[m, i, 2q .. 2q+1] (one 8-byte vector when Np is even, else the j < Np
 *    elements one by one); it stores the pair to Dt[i][q] (one vector);
 *  - u tile: work-item (0,0) copies the tile's rows (one bulk copy, counted
 *    per element); one barrier; when Np is odd every work-item then re-lays
 *    the 128 rows out with pitch 2 Q (row r = lid1 + 16 rb, pair
 *    q = lid0 + XL qb < Q: element loads j < Np, one vector store) and a
 *    second barrier follows;
 *  - for every pair q < Q: vector loads Us[lid1 + 16 a][q] (a < 8) and
 *    Dt[lid0 + XL b][q] (b < NB), 2 x 8 x NB madds (one running sum over the
 *    even j and one over the odd j per output);
 *  - per output (b < NB, a < 8): one add of its two sums, then the store
 *    res[m, k0 + lid1 + 16 a, lid0 + XL b] for k < Nel, i < Np.
 * ====================================================================== */
#define DT_NB(c) (cdiv((c)->P[0], 16))
#define DT_XL(c) (cdiv((c)->P[0], DT_NB(c)))
#define DT_Q(c) (cdiv((c)->P[0], 2))
static long long dt_pd(const ctx *c) { long long p = 2 * DT_Q(c); while (p % 32 != 2) p++; return p; }
static long long ix_dt_D(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0];
    return G0 * Np * Np + (L1_ + 16 * lv[0]) * Np + 2 * (L0_ + DT_XL(c) * lv[1]) + lv[2];
}
static long long ix_dt_D2(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0];
    return (G0 * Np * Np + (L1_ + 16 * lv[0]) * Np) / 2 + L0_ + DT_XL(c) * lv[1];
}
static long long ix_dt_Dt(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return (L1_ + 16 * lv[0]) * (dt_pd(c) / 2) + L0_ + DT_XL(c) * lv[1];
}
static long long ix_dt_u(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)l; return 128 * c->P[0] * G1 + lv[0];
}
static long long ix_dt_R(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return (L1_ + 16 * lv[0]) * c->P[0] + 2 * (L0_ + DT_XL(c) * lv[1]) + lv[2];
}
static long long ix_dt_Ur(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return (L1_ + 16 * lv[0]) * DT_Q(c) + L0_ + DT_XL(c) * lv[1];
}
static long long ix_dt_Us(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return (L1_ + 16 * lv[1]) * DT_Q(c) + lv[0];
}
static long long ix_dt_Dl(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return (L0_ + DT_XL(c) * lv[1]) * (dt_pd(c) / 2) + lv[0];
}
static long long ix_dt_res(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = c->P[0], Nel = c->P[1];
    return G0 * Nel * Np + (128 * G1 + L1_ + 16 * lv[1]) * Np + L0_ + DT_XL(c) * lv[0];
}
/* statements: 0 D vector load, 1 D element load, 2 Dt store, 3 u copy,
 * 4 raw-row element load, 5 re-laid row store, 6 Us load, 7 Dt load,
 * 8 two madds, 9 res store, 10 add of the even-j and odd-j sums */
static void walk_dgt(ctx *c) {
    long long Np = c->P[0], Nel = c->P[1], NB = DT_NB(c), XL = DT_XL(c), Q = DT_Q(c), NPP = XL * NB, lv[3];
    long long k0 = 128 * c->g[1], rows = Nel - k0 < 128 ? Nel - k0 : 128;
    for (lv[0] = 0; lv[0] < cdiv(NPP, 16); lv[0]++)
        for (lv[1] = 0; lv[1] < cdiv(Q, XL); lv[1]++) {
            long long q = c->l[0] + XL * lv[1], i = c->l[1] + 16 * lv[0];
            if (q >= Q || i >= NPP) continue;
            if (i < Np) {
                if (Np % 2 == 0) { lv[2] = 0; X(c, 0, lv); }
                else for (lv[2] = 0; lv[2] < 2; lv[2]++) if (2 * q + lv[2] < Np) X(c, 1, lv);
            }
            X(c, 2, lv);
        }
    if (c->l[0] == 0 && c->l[1] == 0)
        for (lv[0] = 0; lv[0] < rows * Np; lv[0]++) X(c, 3, lv);
    BAR(c);
    if (Np % 2) {
        for (lv[0] = 0; lv[0] < 8; lv[0]++)
            for (lv[1] = 0; lv[1] < cdiv(Q, XL); lv[1]++) {
                long long q = c->l[0] + XL * lv[1];
                if (q >= Q) continue;
                for (lv[2] = 0; lv[2] < 2; lv[2]++) if (2 * q + lv[2] < Np) X(c, 4, lv);
                X(c, 5, lv);
            }
        BAR(c);
    }
    for (lv[0] = 0; lv[0] < Q; lv[0]++) {
        for (lv[1] = 0; lv[1] < 8; lv[1]++) X(c, 6, lv);
        for (lv[1] = 0; lv[1] < NB; lv[1]++) X(c, 7, lv);
        for (lv[1] = 0; lv[1] < 8; lv[1]++)
            for (lv[2] = 0; lv[2] < NB; lv[2]++) X(c, 8, lv);
    }
    for (lv[0] = 0; lv[0] < NB; lv[0]++)
        for (lv[1] = 0; lv[1] < 8; lv[1]++) {
            X(c, 10, lv);
            if (k0 + c->l[1] + 16 * lv[1] < Nel && c->l[0] + XL * lv[0] < Np) X(c, 9, lv);
        }
}
static int setup_dgt(ctx *c) {
    long long Np = c->P[0], Nel = c->P[1];
    if (Np < 1 || Np > 96 || Nel < 4 || Nel % 4 || Nel > 65535LL * 128) return -1;
    c->grid[0] = 3; c->grid[1] = cdiv(Nel, 128); c->grid[2] = 1;
    c->wg[0] = DT_XL(c); c->wg[1] = 16; c->wg[2] = 1;
    int s0 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "dgt-D", MEM_GLOBAL, DIR_LOAD, "float32x2", 8, ix_dt_D2));
    int s1 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s1, add_site(c, "dgt-D", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dt_D));
    int s2 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s2, add_site(c, "dgt-Dt", MEM_LOCAL, DIR_STORE, "float32x2", 8, ix_dt_Dt));
    int s3 = add_stmt(c, 1, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "dgt-u", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dt_u));
    int s4 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s4, add_site(c, "dgt-R", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_dt_R));
    int s5 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s5, add_site(c, "dgt-Ur", MEM_LOCAL, DIR_STORE, "float32x2", 8, ix_dt_Ur));
    int s6 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s6, add_site(c, "dgt-Us", MEM_LOCAL, DIR_LOAD, "float32x2", 8, ix_dt_Us));
    int s7 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s7, add_site(c, "dgt-Dl", MEM_LOCAL, DIR_LOAD, "float32x2", 8, ix_dt_Dl));
    add_stmt(c, 3, DT_F32, 0, 0, 2);
    int s9 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s9, add_site(c, "dgt-res", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dt_res));
    add_stmt(c, 2, DT_F32, 1, 0, 0);
    c->walk = walk_dgt;
    return 0;
}

/* ======================================================================
 * DG derivative on the tensor cores ("dg_tc"), res[m, k, i] =
 * sum_j D[m, i, j] u[k, j], TF32 head/remainder split in three passes.
 * P = {Np, Nel, P, A}.  Np in {4, 10, 20, 35, 56, 84}; Nel a multiple of 4.
 * The kernel's definition of its launch:
 *   A < 0 means A = 1 for 20 < Np <= 40 and for Np > 64, else 0;
 *   MS = 3 m per work-group for Np <= 40 and, with A = 0, for Np <= 64,
 *   else 1; G = 3 / MS m-groups; R = 2 work-groups per SM for A = 0 and
 *   Np <= 20, else 1; P = 0 means min(T, 152 R / G), T = ceil(Nel / 128);
 *   grid (G, P), work-group of 320 work-items (1-D), 352 for A = 1.
 * NP8 = Np rounded up to 8, NR = MS NP8 rounded up to 16 (MMA N), KA =
 * ceil(Np / 32) atoms of 32 columns, KS = ceil(Np / 8) k steps, CN(a) =
 * 2 min(4, KS - 4a) chunks of atom a.  Work-group (g, p) serves tiles
 * t = p + P lt < T; rows(t) = min(128, Nel - 128 t).  Per work-item tid:
 *  - tid < NP8, m-block mm < MS, chunk ac < 8 KA: element loads
 *    D[m, tid, 4 ac + x] (m = mm when MS = 3, else g) for tid, 4 ac + x < Np;
 *    one statement with 4 adds and two 16-byte local stores (head,
 *    remainder) at row mm NP8 + tid, chunk ac;
 *  - tid < NR - MS NP8: two zero stores per chunk ac of padding row
 *    MS NP8 + tid;  one barrier;
 *  - per tile, Np % 4 == 0: work-item 256 copies element (r, cc) of the box
 *    at row 128 t, column 32 a for r < rows(t), 32 a + cc < Np;
 *  - per tile, Np % 4 != 0 and A = 1: work-item 256 copies the tile's
 *    rows(t) x Np elements of u (one bulk copy);
 *  - per tile, converter 128 <= tid < 256, r = tid - 128, atom a, chunk
 *    c < CN(a): Np % 4 == 0: a 16-byte local load of (r, c); else element
 *    loads of u[128 t + r, 32 a + 4 c + x] (from the staged rows, local, for
 *    A = 1; from global memory for A = 0) for 128 t + r < Nel,
 *    32 a + 4 c + x < Np; one statement of 4 adds with, for A = 0, two
 *    16-byte local stores (r, c);
 *  - per tile, work-item 288 (A = 1: 288 for the work-group's even-numbered
 *    tiles lt, 320 for the odd ones), atom a, k step kk < min(4, KS - 4a):
 *    3 x 128 x NR x 8 TF32 multiply-adds;
 *  - per tile, epilogue tid < 128, per m-block mm: the row's Np / 4 16-byte
 *    local stores (Np % 4 == 0, else Np element stores), and work-item 0
 *    stores the rows(t) x Np elements of res[m, 128 t .., :] (m = mm when
 *    MS = 3, else g);
 *  - two barriers at the end.
 * The epilogue's own synchronisation (named barriers over its 128
 * work-items) is not a work-group barrier and is not counted: every
 * work-item passes the same three work-group barriers.
 * Local sites are indexed by the logical (row, chunk) position in one ring
 * stage or staging buffer.
 * ====================================================================== */
#define DC_NP(c) ((c)->P[0])
#define DC_MS(c) ((c)->D[1])
#define DC_NP8(c) ((DC_NP(c) + 7) / 8 * 8)
#define DC_NR(c) ((DC_MS(c) * DC_NP8(c) + 15) / 16 * 16)
#define DC_KA(c) (cdiv(DC_NP(c), 32))
#define DC_KS(c) (cdiv(DC_NP(c), 8))
static long long dc_m(const ctx *c, const long long *g, long long mm) { return DC_MS(c) == 3 ? mm : G0; }
static long long dc_tile(const ctx *c, const long long *g, long long lt) { return G1 + c->D[0] * lt; }
static long long ix_dc_D(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = DC_NP(c);
    return (dc_m(c, g, lv[0]) * Np + L0_) * Np + 4 * lv[1] + lv[2];
}
static long long ix_dc_B(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return (lv[0] * DC_NP8(c) + L0_) * 8 * DC_KA(c) + lv[1];
}
static long long ix_dc_ubox(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)l; long long Np = DC_NP(c), a = lv[1] / 128, r = lv[1] % 128;
    return (128 * dc_tile(c, g, lv[0]) + r) * Np + 32 * a + lv[2];
}
static long long ix_dc_ug(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    long long Np = DC_NP(c);
    return (128 * dc_tile(c, g, lv[0]) + (L0_ - 128)) * Np + 4 * lv[1] + lv[2];
}
static long long ix_dc_ubulk(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)l; return 128 * dc_tile(c, g, lv[0]) * DC_NP(c) + lv[1];
}
static long long ix_dc_R(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; return (L0_ - 128) * DC_NP(c) + 4 * lv[1] + lv[2];
}
static long long ix_dc_U(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; (void)c; return (L0_ - 128) * 8 + lv[2];
}
static long long ix_dc_O(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)g; long long Np = DC_NP(c); return L0_ * (Np % 4 == 0 ? Np / 4 : Np) + lv[2];
}
static long long ix_dc_res(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)l; long long Np = DC_NP(c), Nel = c->P[1];
    return (dc_m(c, g, lv[1]) * Nel + 128 * dc_tile(c, g, lv[0])) * Np + lv[2];
}
/* statements: 0 D element load, 1 split + operator stores, 2 padding stores,
 * 3 u box element copy, 4 u element load, 5 staged-chunk load, 6 split (+
 * stores for A = 0), 7 MMA k step, 8 staging store, 9 res element copy,
 * 10 u tile element copy (bulk), 11 staged-row element load */
static void walk_dgc(ctx *c) {
    long long Np = DC_NP(c), Nel = c->P[1], P = c->D[0], MS = DC_MS(c), NP8 = DC_NP8(c), NR = DC_NR(c);
    long long KA = DC_KA(c), KS = DC_KS(c), T = cdiv(Nel, 128), tid = c->l[0], lv[3];
    if (tid < NP8)
        for (lv[0] = 0; lv[0] < MS; lv[0]++)
            for (lv[1] = 0; lv[1] < 8 * KA; lv[1]++) {
                for (lv[2] = 0; lv[2] < 4; lv[2]++)
                    if (tid < Np && 4 * lv[1] + lv[2] < Np) X(c, 0, lv);
                X(c, 1, lv);
            }
    if (tid < NR - MS * NP8) {
        lv[0] = MS;
        for (lv[1] = 0; lv[1] < 8 * KA; lv[1]++) X(c, 2, lv);
    }
    BAR(c);
    for (long long lt = 0; c->g[1] + P * lt < T; lt++) {
        const long long t = c->g[1] + P * lt, rows = Nel - 128 * t < 128 ? Nel - 128 * t : 128;
        lv[0] = lt;
        if (tid == 256 && Np % 4 != 0 && c->D[2])
            for (lv[1] = 0; lv[1] < rows * Np; lv[1]++) X(c, 10, lv);
        if (tid == 256 && Np % 4 == 0)
            for (long long a = 0; a < KA; a++)
                for (long long r = 0; r < rows; r++) {
                    lv[1] = 128 * a + r;
                    for (lv[2] = 0; lv[2] < 32 && 32 * a + lv[2] < Np; lv[2]++) X(c, 3, lv);
                }
        if (tid >= 128 && tid < 256) {
            const long long r = tid - 128;
            for (long long a = 0; a < KA; a++) {
                const long long cn = 2 * (KS - 4 * a < 4 ? KS - 4 * a : 4);
                for (long long ch = 0; ch < cn; ch++) {
                    if (Np % 4 == 0) {
                        lv[1] = a; lv[2] = ch;
                        X(c, 5, lv);
                    } else {
                        lv[1] = 8 * a + ch;
                        for (lv[2] = 0; lv[2] < 4; lv[2]++)
                            if (128 * t + r < Nel && 32 * a + 4 * ch + lv[2] < Np) X(c, c->D[2] ? 11 : 4, lv);
                    }
                    lv[1] = a; lv[2] = ch;
                    X(c, 6, lv);
                }
            }
        }
        if (tid == (c->D[3] && (lt & 1) ? 320 : 288))
            for (lv[1] = 0; lv[1] < KA; lv[1]++)
                for (lv[2] = 0; lv[2] < 4 && 4 * lv[1] + lv[2] < KS; lv[2]++) X(c, 7, lv);
        if (tid < 128) {
            for (lv[1] = 0; lv[1] < MS; lv[1]++) {
                for (lv[2] = 0; lv[2] < (Np % 4 == 0 ? Np / 4 : Np); lv[2]++) X(c, 8, lv);
                if (tid == 0)
                    for (lv[2] = 0; lv[2] < rows * Np; lv[2]++) X(c, 9, lv);
            }
        }
    }
    BAR(c);
    BAR(c);
    (void)NR;
}
static int setup_dgc(ctx *c) {
    long long Np = DC_NP(c), Nel = c->P[1], P = c->P[2], A = c->P[3];
    if (Np != 4 && Np != 10 && Np != 20 && Np != 35 && Np != 56 && Np != 84) return -1;
    if (Nel < 4 || Nel % 4 || P < 0 || A < -1 || A > 1) return -1;
    if (A < 0) A = (Np > 20 && Np <= 40) || Np > 64;
    c->D[1] = (Np <= 40 || (A == 0 && Np <= 64)) ? 3 : 1;
    c->D[2] = (A == 1 && Np % 4 != 0);   /* u tiles by one bulk copy each */
    c->D[3] = A;                          /* A = 1: two MMA work-items, alternate tiles */
    const long long MS = DC_MS(c), G = 3 / MS, R = (A == 0 && Np <= 20) ? 2 : 1, T = cdiv(Nel, 128);
    if (P == 0) P = T < 152 * R / G ? T : 152 * R / G;
    c->D[0] = P;
    c->grid[0] = G; c->grid[1] = P; c->grid[2] = 1;
    c->wg[0] = A == 1 ? 352 : 320; c->wg[1] = 1; c->wg[2] = 1;
    const int tf = (Np % 4 == 0);
    int s0 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s0, add_site(c, "dgc-D", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dc_D));
    int sBh = add_site(c, "dgc-Bh", MEM_LOCAL, DIR_STORE, "float32x4", 16, ix_dc_B);
    int sBl = add_site(c, "dgc-Bl", MEM_LOCAL, DIR_STORE, "float32x4", 16, ix_dc_B);
    int s1 = add_stmt(c, 2, DT_F32, 4, 0, 0);
    stmt_site(c, s1, sBh); stmt_site(c, s1, sBl);
    int s2 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s2, sBh); stmt_site(c, s2, sBl);
    int s3 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s3, add_site(c, "dgc-u", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dc_ubox));
    int s4 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s4, add_site(c, "dgc-u", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dc_ug));
    int s5 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s5, add_site(c, "dgc-Ur", MEM_LOCAL, DIR_LOAD, "float32x4", 16, ix_dc_U));
    int s6 = add_stmt(c, 3, DT_F32, 4, 0, 0);
    if (A == 0) {
        stmt_site(c, s6, add_site(c, "dgc-Uh", MEM_LOCAL, DIR_STORE, "float32x4", 16, ix_dc_U));
        stmt_site(c, s6, add_site(c, "dgc-Ul", MEM_LOCAL, DIR_STORE, "float32x4", 16, ix_dc_U));
    }
    add_stmt(c, 3, DT_TF32, 0, 0, (int)(3 * 128 * DC_NR(c) * 8));
    int s8 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s8, add_site(c, "dgc-O", MEM_LOCAL, DIR_STORE, tf ? "float32x4" : "float32", tf ? 16 : 4, ix_dc_O));
    int s9 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s9, add_site(c, "dgc-res", MEM_GLOBAL, DIR_STORE, "float32", 4, ix_dc_res));
    int s10 = add_stmt(c, 2, DT_F32, 0, 0, 0);
    stmt_site(c, s10, add_site(c, "dgc-u", MEM_GLOBAL, DIR_LOAD, "float32", 4, ix_dc_ubulk));
    int s11 = add_stmt(c, 3, DT_F32, 0, 0, 0);
    stmt_site(c, s11, add_site(c, "dgc-R", MEM_LOCAL, DIR_LOAD, "float32", 4, ix_dc_R));
    (void)s0; (void)s3; (void)s4; (void)s5; (void)s10; (void)s11;
    c->walk = walk_dgc;
    return 0;
}

/* ======================================================================
 * Public oracle entry: enumerate every (group, sub-group, lane) point.
 * ====================================================================== */
typedef struct {
    int kind;                 /* 0 op, 1 mem access site, 2 barrier, 3 groups, 4 launch, 5 grid */
    char name[24];            /* op: "add"/"mul"/"madd"; site: tag */
    char dtype[16];
    int mem, dir, dsize, uniform, affine;
    long long lstr[3], gstr[3], loopstr;
    unsigned long long wi, sg, footprint;
} orec;

/* ======================================================================
 * Work removal (Algorithm 3) on a parent descriptor: every statement is
 * replaced by one "tgt = tgt + load" statement (one add) per global load it
 * contains that is not in the removal set, and by "store = tgt" for a kept
 * global store, at the same loop point and under the same guards; local
 * memory accesses, arithmetic and barriers go.  If no global store is kept,
 * every work-item finally writes tgt to its own entry of tgt_dest
 * (row-major over the global index space).
 * ====================================================================== */
static long long ix_tgt_dest(const ctx *c, const long long *g, const long long *l, const long long *lv) {
    (void)lv;
    const long long L0 = c->wg[0], L1 = c->wg[1], L2 = c->wg[2];
    return ((g[2] * L2 + l[2]) * (c->grid[1] * L1) + g[1] * L1 + l[1]) * (c->grid[0] * L0) + g[0] * L0 + l[0];
}
static int make_twin(ctx *c, const char *remove) {
    /* remove: tags separated by '|' */
    const int nst = c->nstmt;
    int kept_store = 0, first_dt = -1;
    const char *dname = "float32";
    int dsize = 4;
    for (int st = 0; st < nst; st++) {
        stmt_t S = c->stmt[st];
        c->tmap_n[st] = 0;
        for (int a = 0; a < S.nsite; a++) {
            const site_t *x = &c->site[S.site[a]];
            if (x->mem != MEM_GLOBAL) continue;
            char key[64];
            snprintf(key, sizeof key, "|%s|", x->tag);
            char all[1024];
            snprintf(all, sizeof all, "|%s|", remove);
            if (strstr(all, key)) continue;
            if (c->nstmt >= MAXSTMT || c->tmap_n[st] >= 8) return -1;
            int t = add_stmt(c, S.nloop, S.dt, x->dir == DIR_LOAD ? 1 : 0, 0, 0);
            stmt_site(c, t, S.site[a]);
            c->tmap[st][c->tmap_n[st]++] = t;
            if (x->dir == DIR_STORE) kept_store = 1;
            else if (first_dt < 0) { first_dt = S.dt; dname = x->dtype; dsize = x->dsize; }
        }
    }
    c->tdest = -1;
    if (!kept_store) {
        if (c->nstmt >= MAXSTMT || c->nsite >= MAXSITE) return -1;
        c->tdest = add_stmt(c, 0, first_dt < 0 ? DT_F32 : first_dt, 0, 0, 0);
        stmt_site(c, c->tdest, add_site(c, "tgt_dest", MEM_GLOBAL, DIR_STORE, dname, dsize, ix_tgt_dest));
    }
    c->twin = 1;
    return 0;
}

static const struct { const char *name; int fam, v; } KTAB[] = {
    {"stream", 0, 0}, {"fma", 1, 0}, {"smem", 2, 0}, {"barrier", 3, 0}, {"overlap", 4, 0}, {"empty", 5, 0},
    {"mm_pf", 6, 0}, {"mm_nopf", 6, 1}, {"mm_pf_a", 6, 2}, {"mm_pf_b", 6, 3}, {"mm_nopf_a", 6, 4}, {"mm_nopf_b", 6, 5},
    {"dg_nopf", 7, 0}, {"dg_dmpf", 7, 1}, {"dg_nopf_u", 7, 2}, {"dg_nopf_dm", 7, 3}, {"dg_dmpf_u", 7, 4},
    {"dg_dmpf_dm", 7, 5}, {"dg_res", 7, 6},
    {"fd_tile", 8, 0}, {"fd_direct", 8, 1}, {"fd_tile_u", 8, 2}, {"fd_tile_res", 8, 3}, {"fd_direct_u", 8, 4},
    {"fd_direct_res", 8, 5}, {"fd_tile18", 8, 6}, {"fd_tile18_u", 8, 7}, {"fd_tile18_res", 8, 8},
    {"dg_upf", 7, 7}, {"dg_dmpft", 7, 8}, {"dg_upf_u", 7, 9}, {"dg_dmpft_u", 7, 10}, {"dg_dmpft_res", 7, 11},
    {"mm_simt", 9, 0},
    {"mm_tc", 10, 0},
    {"fd_block", 11, 0},
    {"smem2d", 12, 0},
    {"mm_tc256", 10, 1},
    {"dg_tile", 13, 0},
    {"dg_tc", 14, 0},
};

static int counts_impl(const char *kernel, const char *remove, const long long *P, int nP, orec *out, int cap,
                       int *n_out);
int oracle_counts(const char *kernel, const long long *P, int nP, orec *out, int cap, int *n_out) {
    return counts_impl(kernel, NULL, P, nP, out, cap, n_out);
}
/* counts of the work-removed twin of `kernel` (Algorithm 3), global accesses
 * whose tags are listed in `remove` ('|'-separated) removed */
int oracle_counts_twin(const char *kernel, const char *remove, const long long *P, int nP, orec *out, int cap,
                       int *n_out) {
    return counts_impl(kernel, remove ? remove : "", P, nP, out, cap, n_out);
}
static int counts_impl(const char *kernel, const char *remove, const long long *P, int nP, orec *out, int cap,
                       int *n_out) {
    ctx *c = (ctx *)calloc(1, sizeof(ctx));
    int fam = -1, v = 0, rc = 0;
    for (size_t i = 0; i < sizeof KTAB / sizeof KTAB[0]; i++)
        if (!strcmp(KTAB[i].name, kernel)) { fam = KTAB[i].fam; v = KTAB[i].v; }
    if (fam < 0 || nP > 8) { free(c); return -1; }
    for (int i = 0; i < nP; i++) c->P[i] = P[i];
    switch (fam) {
    case 0: rc = setup_stream(c); break;
    case 1: rc = setup_fma(c); break;
    case 2: rc = setup_smem(c); break;
    case 3: rc = setup_barrier(c); break;
    case 4: rc = setup_overlap(c); break;
    case 5: rc = setup_empty(c); break;
    case 6: rc = setup_mm(c, v); break;
    case 7: rc = setup_dg(c, v); break;
    case 8: rc = setup_fd(c, v); break;
    case 9: rc = setup_simt(c); break;
    case 10: rc = v ? setup_tcw(c) : setup_tc(c); break;
    case 11: rc = setup_fdb(c); break;
    case 12: rc = setup_smem2d(c); break;
    case 13: rc = setup_dgt(c); break;
    case 14: rc = setup_dgc(c); break;
    }
    if (rc) { free(c); return -2; }
    if (remove && make_twin(c, remove)) { free(c); return -5; }
    for (int s = 0; s < c->nsite; s++) ks_init(&c->ss[s].foot, 1024);
    ks_init(&c->sgset, 1024);
    c->bar_min = -1; c->bar_max = -1;
    long long L0 = c->wg[0], L1 = c->wg[1], L2 = c->wg[2], T = L0 * L1 * L2;
    long long g[3];
    for (g[2] = 0; g[2] < c->grid[2]; g[2]++)
    for (g[1] = 0; g[1] < c->grid[1]; g[1]++)
    for (g[0] = 0; g[0] < c->grid[0]; g[0]++) {
        for (long long q = 0; q * SGSIZE < T; q++) {
            ks_clear(&c->sgset);
            for (long long lane = 0; lane < SGSIZE && q * SGSIZE + lane < T; lane++) {
                long long t = q * SGSIZE + lane;
                c->g[0] = g[0]; c->g[1] = g[1]; c->g[2] = g[2];
                c->l[0] = t % L0; c->l[1] = (t / L0) % L1; c->l[2] = t / (L0 * L1);
                c->bar_cur = 0;
                c->walk(c);
                if (c->twin && c->tdest >= 0) X_exec(c, c->tdest, NULL);
                if (c->bar_min < 0 || c->bar_cur < c->bar_min) c->bar_min = c->bar_cur;
                if (c->bar_cur > c->bar_max) c->bar_max = c->bar_cur;
            }
        }
    }
    if (c->err) { rc = -3; goto done; }
    int n = 0;
#define EMIT() do { if (n >= cap) { rc = -4; goto done; } memset(&out[n], 0, sizeof(orec)); } while (0)
    static const char *opn[3] = {"add", "mul", "madd"};
    static const char *dtn[4] = {"float32", "float64", "bfloat16", "tfloat32"};
    for (int dt = 0; dt < 4; dt++)
        for (int o = 0; o < 3; o++)
            if (c->op_wi[dt][o]) {
                EMIT();
                out[n].kind = 0;
                strcpy(out[n].name, opn[o]);
                strcpy(out[n].dtype, dtn[dt]);
                out[n].wi = c->op_wi[dt][o]; out[n].sg = c->op_sg[dt][o];
                n++;
            }
    for (int s = 0; s < c->nsite; s++) {
        if (c->ss[s].wi == 0) continue;
        EMIT();
        orec *r = &out[n++];
        r->kind = 1;
        strncpy(r->name, c->site[s].tag, sizeof r->name - 1);
        strncpy(r->dtype, c->site[s].dtype, sizeof r->dtype - 1);
        r->mem = c->site[s].mem; r->dir = c->site[s].dir; r->dsize = c->site[s].dsize;
        for (int a = 0; a < 3; a++) { r->lstr[a] = c->ss[s].lstr[a]; r->gstr[a] = c->ss[s].gstr[a]; }
        r->loopstr = c->ss[s].loopstr;
        r->affine = c->ss[s].affine;
        r->uniform = r->lstr[0] == 0;
        r->wi = c->ss[s].wi; r->sg = c->ss[s].sg; r->footprint = c->ss[s].foot.n;
    }
    EMIT(); out[n].kind = 2; strcpy(out[n].name, "barrier_local");
    out[n].wi = (unsigned long long)(c->bar_max < 0 ? 0 : c->bar_max);
    out[n].sg = (unsigned long long)(c->bar_min < 0 ? 0 : c->bar_min); n++;
    EMIT(); out[n].kind = 3; strcpy(out[n].name, "thread_groups");
    out[n].wi = (unsigned long long)(c->grid[0] * c->grid[1] * c->grid[2]); n++;
    EMIT(); out[n].kind = 4; strcpy(out[n].name, "kernel_launch"); out[n].wi = 1; n++;
    EMIT(); out[n].kind = 5; strcpy(out[n].name, "grid");
    for (int a = 0; a < 3; a++) { out[n].lstr[a] = c->wg[a]; out[n].gstr[a] = c->grid[a]; }
    n++;
    *n_out = n;
done:
    for (int s = 0; s < c->nsite; s++) ks_free(&c->ss[s].foot);
    ks_free(&c->sgset);
    free(c);
    return rc;
}

int oracle_sizeof_orec(void) { return (int)sizeof(orec); }

/* ======================================================================
 * Reference outputs.  FP64 references follow the mathematical definition;
 * bit-exact replays follow the kernel definition's operation order (this
 * file is compiled with -ffp-contract=off so no multiply-add is fused
 * unless fma()/fmaf() is called explicitly).
 * ====================================================================== */

/* stream: out[e] = ((in0[e] + in1[e]) + in2[e]) + ..., in the kernel's dtype */
void oracle_stream_ref(int dtype, int L, long long N, const void *const *ins, void *out) {
    if (dtype == DT_F32) {
        const float *const *x = (const float *const *)ins; float *o = (float *)out;
        for (long long e = 0; e < N; e++) { float s = x[0][e]; for (int a = 1; a < L; a++) s = s + x[a][e]; o[e] = s; }
    } else {
        const double *const *x = (const double *const *)ins; double *o = (double *)out;
        for (long long e = 0; e < N; e++) { double s = x[0][e]; for (int a = 1; a < L; a++) s = s + x[a][e]; o[e] = s; }
    }
}

/* arithmetic kernel constants (the kernel's definition):
 *   x_t = u + t/32;  add: x += 2^-13;  mul: x *= 1 - 2^-12;
 *   madd: x = x*(1 - 2^-10) + 2^-10;   out = x_0 + x_1 + ... + x_31 */
void oracle_fma_ref(int dtype, int op, long long F, long long nthreads, const void *seed, void *out) {
    long long R = F / 32;
    if (dtype == DT_F32) {
        const float *u = (const float *)seed; float *o = (float *)out;
        const float ca = 0.0001220703125f, ma = 0.999755859375f, fa = 0.9990234375f, fb = 0.0009765625f;
        for (long long t = 0; t < nthreads; t++) {
            float x[32];
            for (int k = 0; k < 32; k++) x[k] = u[t] + (float)k * 0.03125f;
            for (long long r = 0; r < R; r++)
                for (int k = 0; k < 32; k++) {
                    if (op == 0) x[k] = x[k] + ca;
                    else if (op == 1) x[k] = x[k] * ma;
                    else x[k] = fmaf(x[k], fa, fb);
                }
            float s = x[0];
            for (int k = 1; k < 32; k++) s = s + x[k];
            o[t] = s;
        }
    } else {
        const double *u = (const double *)seed; double *o = (double *)out;
        const double ca = 0.0001220703125, ma = 0.999755859375, fa = 0.9990234375, fb = 0.0009765625;
        for (long long t = 0; t < nthreads; t++) {
            double x[32];
            for (int k = 0; k < 32; k++) x[k] = u[t] + (double)k * 0.03125;
            for (long long r = 0; r < R; r++)
                for (int k = 0; k < 32; k++) {
                    if (op == 0) x[k] = x[k] + ca;
                    else if (op == 1) x[k] = x[k] * ma;
                    else x[k] = fma(x[k], fa, fb);
                }
            double s = x[0];
            for (int k = 1; k < 32; k++) s = s + x[k];
            o[t] = s;
        }
    }
}

/* matmul FP64 reference and the per-element absolute-value sum sum_k |a_ik b_kj| */
void oracle_mm_ref(long long n, const float *a, const float *b, double *c, double *cabs) {
    for (long long i = 0; i < n; i++)
        for (long long j = 0; j < n; j++) {
            double s = 0.0, sa = 0.0;
            for (long long k = 0; k < n; k++) {
                double p = (double)a[n * i + k] * (double)b[n * k + j];
                s += p; sa += fabs(p);
            }
            c[n * i + j] = s; cabs[n * i + j] = sa;
        }
}

/* DG FP64 reference: res[m,k,i] = sum_j D[m,i,j] u[k,j] (and |.| sums) */
void oracle_dg_ref(long long Np, long long Nel, const float *D, const float *u, double *res, double *rabs) {
    for (long long m = 0; m < 3; m++)
        for (long long k = 0; k < Nel; k++)
            for (long long i = 0; i < Np; i++) {
                double s = 0.0, sa = 0.0;
                for (long long j = 0; j < Np; j++) {
                    double p = (double)D[Np * Np * m + Np * i + j] * (double)u[Np * k + j];
                    s += p; sa += fabs(p);
                }
                res[Nel * Np * m + Np * k + i] = s; rabs[Nel * Np * m + Np * k + i] = sa;
            }
}

/* stencil FP64 reference on an (h+2) x (n+2) input -> h x n output */
void oracle_fd_ref(long long h, long long n, double c0, double c1, const float *u, double *res, double *rabs) {
    long long W = n + 2;
    for (long long i = 0; i < h; i++)
        for (long long j = 0; j < n; j++) {
            double C = u[W * (i + 1) + j + 1], N_ = u[W * i + j + 1], S = u[W * (i + 2) + j + 1];
            double Wv = u[W * (i + 1) + j], E = u[W * (i + 1) + j + 2];
            res[n * i + j] = c0 * C + c1 * (N_ + S + Wv + E);
            rabs[n * i + j] = fabs(c0 * C) + fabs(c1) * (fabs(N_) + fabs(S) + fabs(Wv) + fabs(E));
        }
}

/* bit-exact FP32 replay of the work-removed (gmem-only) twins: each work-item
 * sums its loads sequentially, starting from 0.0f, in loop order. */
void oracle_mm_twin_ref(int v, long long n, const float *x, float *dest) {
    /* v: 2 PF-a, 3 PF-b, 4 noPF-a, 5 noPF-b; dest is n x n (one entry per WI) */
    for (long long i = 0; i < n; i++)
        for (long long j = 0; j < n; j++) {
            float t = 0.0f;
            long long g0 = j / 16, l0 = j % 16, g1 = i / 16, l1 = i % 16;
            if (v == 2) for (long long ko = 0; ko < n / 16; ko++) t = t + x[n * (16 * g1 + l1) + 16 * ko + l0];
            if (v == 3) for (long long ko = 0; ko < n / 16; ko++) t = t + x[n * (16 * ko + l1) + 16 * g0 + l0];
            if (v == 4) for (long long k = 0; k < n; k++) t = t + x[n * i + k];
            if (v == 5) for (long long k = 0; k < n; k++) t = t + x[n * k + j];
            dest[n * i + j] = t;
        }
}

void oracle_dg_twin_ref(int v, long long Np, long long Nel, long long L0, long long L1, const float *D,
                        const float *u, float *dest) {
    /* v: 2 noPF-u, 3 noPF-dm, 4 dmPF-u, 5 dmPF-dm, 9 uPF-u, 10 dmPF-T-u (u given
     * as uT[j, k]); dest rows = ceil(Np/L1)*L1, cols = Nel */
    long long rows = cdiv(Np, L1) * L1, nj = cdiv(Np, L0), njl = cdiv(Np, L1);
    for (long long i = 0; i < rows; i++)
        for (long long k = 0; k < Nel; k++) {
            float t = 0.0f;
            long long l0 = k % L0;
            if (v == 9)   /* every work-item fetches, whatever its row i */
                for (long long jo = 0; jo < njl; jo++)
                    if (L1 * jo + l0 < Np) t = t + u[Np * (L0 * (k / L0) + i % L1) + L1 * jo + l0];
            if (i < Np) for (long long m = 0; m < 3; m++) {
                if (v == 10) for (long long j = 0; j < Np; j++) t = t + u[Nel * j + k];
                if (v == 2 || v == 4) for (long long j = 0; j < Np; j++) t = t + u[Np * k + j];
                if (v == 3) for (long long j = 0; j < Np; j++) t = t + D[Np * Np * m + Np * i + j];
                if (v == 5) for (long long jo = 0; jo < nj; jo++)
                    if (L0 * jo + l0 < Np) t = t + D[Np * Np * m + Np * i + L0 * jo + l0];
            }
            dest[Nel * i + k] = t;
        }
}

void oracle_fd_twin_ref(int v, long long n, const float *u, float *dest) {
    /* v: 2 tile-u (dest is (16*G1) x (16*G0), G = ceil(n/14)),
     *    7 tile18-u (dest is (18*G1) x (18*G0), G = ceil(n/16)),
     *    4 direct-u (dest is (16*G1) x (16*G0), G = ceil(n/16)) */
    long long W = n + 2;
    if (v == 2 || v == 7) {
        long long T = v == 2 ? 16 : 18, G = cdiv(n, T - 2), cols = T * G;
        for (long long gi = 0; gi < G; gi++) for (long long gj = 0; gj < G; gj++)
        for (long long l1 = 0; l1 < T; l1++) for (long long l0 = 0; l0 < T; l0++) {
            long long r = (T - 2) * gi + l1, q = (T - 2) * gj + l0;
            float t = 0.0f;
            if (r < W && q < W) t = t + u[W * r + q];
            dest[cols * (T * gi + l1) + T * gj + l0] = t;
        }
    } else {
        long long G = cdiv(n, 16), cols = 16 * G;
        for (long long i = 0; i < 16 * G; i++) for (long long j = 0; j < 16 * G; j++) {
            float t = 0.0f;
            if (i < n && j < n) {
                t = t + u[W * (i + 1) + j + 1];
                t = t + u[W * i + j + 1];
                t = t + u[W * (i + 2) + j + 1];
                t = t + u[W * (i + 1) + j];
                t = t + u[W * (i + 1) + j + 2];
            }
            dest[cols * i + j] = t;
        }
    }
}

/* worked example of Section "Gathering Kernel Statistics": number of integer
 * points (i, j) with p <= i < n and p <= j < i + 1, by brute force. */
long long oracle_count_example(long long n, long long p) {
    long long cnt = 0;
    for (long long i = p; i < n; i++)
        for (long long j = p; j < i + 1; j++) cnt++;
    return cnt;
}
