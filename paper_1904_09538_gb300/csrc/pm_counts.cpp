// Exact kernel features in closed form (Algorithm 1: count = sum over
// statements of |projection of the loop domain| x operations per instance;
// Algorithm 2 per access site for the footprint; granularities of Section
// "Gathering Kernel Statistics": sub-group = 32 consecutive linear ids,
// on-chip work and uniform global accesses per sub-group, other global
// accesses per work-item, barriers per work-item).
//
// Each kernel's loop domain is the one its CUDA kernel executes; the
// formulas below count that domain's statement instances directly.
#include <algorithm>
#include <cstring>

#include "pm_internal.h"

namespace pm {

namespace {

typedef unsigned long long u64;
typedef long long i64;

i64 cdiv(i64 a, i64 b) { return (a + b - 1) / b; }

pm_feature op_rec(const char *dtype, const char *op, u64 wi, u64 sg) {
    pm_feature f;
    memset(&f, 0, sizeof f);
    f.kind = PM_FEAT_OP;
    f.gran = PM_GRAN_SG;
    f.count = sg;
    f.count_wi = wi;
    f.count_sg = sg;
    snprintf(f.dtype, sizeof f.dtype, "%s", dtype);
    snprintf(f.op, sizeof f.op, "%s", op);
    return f;
}

struct Site {
    const char *tag;
    int mem, dir;
    const char *dtype;
    int dsize;
    int nl;
    i64 l[3];
    int ng;
    i64 g[3];
    i64 loop;
    u64 wi, sg, foot;
};

pm_feature mem_rec(const Site &s) {
    pm_feature f;
    memset(&f, 0, sizeof f);
    f.kind = PM_FEAT_MEM;
    snprintf(f.tag, sizeof f.tag, "%s", s.tag);
    snprintf(f.dtype, sizeof f.dtype, "%s", s.dtype);
    f.mem = s.mem;
    f.dir = s.dir;
    f.dsize = s.dsize;
    f.nl = s.nl;
    f.ng = s.ng;
    for (int a = 0; a < 3; a++) {
        f.lstride[a] = s.l[a];
        f.gstride[a] = s.g[a];
    }
    f.loop_stride = s.loop;
    f.count_wi = s.wi;
    f.count_sg = s.sg;
    f.accesses = s.wi;
    f.footprint = s.foot;
    bool per_sg = s.mem == 1 || s.l[0] == 0;
    f.gran = per_sg ? PM_GRAN_SG : PM_GRAN_WI;
    f.count = per_sg ? s.sg : s.wi;
    return f;
}

pm_feature simple(int kind, int gran, u64 c) {
    pm_feature f;
    memset(&f, 0, sizeof f);
    f.kind = kind;
    f.gran = gran;
    f.count = c;
    return f;
}

struct Out {
    std::vector<pm_feature> &v;
    // op totals in the enumeration order float32 add, mul, madd, float64 add, mul, madd
    u64 wi[2][3] = {{0}}, sg[2][3] = {{0}};
    std::vector<pm_feature> sites;
    explicit Out(std::vector<pm_feature> &o) : v(o) {}
    void op(int dt, int o, u64 w, u64 s) { wi[dt][o] += w; sg[dt][o] += s; }
    void site(const Site &s) {
        if (s.wi) sites.push_back(mem_rec(s));
    }
    void finish(u64 barriers, u64 groups) {
        static const char *on[3] = {"add", "mul", "madd"};
        for (int dt = 0; dt < 2; dt++)
            for (int o = 0; o < 3; o++)
                if (wi[dt][o]) v.push_back(op_rec(dt ? "float64" : "float32", on[o], wi[dt][o], sg[dt][o]));
        for (auto &s : sites) v.push_back(s);
        v.push_back(simple(PM_FEAT_SYNC, PM_GRAN_WI, barriers));
        v.push_back(simple(PM_FEAT_GROUPS, PM_GRAN_WG, groups));
        v.push_back(simple(PM_FEAT_LAUNCH, PM_GRAN_K, 1));
    }
};

const int GL = 0, LO = 1, LD = 0, ST = 1;

// ---------------------------------------------------------------- stream
int stream_width(i64 dt, i64 vec) { return vec ? (dt == 0 ? 4 : 2) : 1; }

pm_status counts_stream(const KP &kp, std::vector<pm_feature> &v) {
    i64 dt = kp.i(0), vec = kp.i(1), N = kp.i(2), s = kp.i(3), L = kp.i(4), shape = kp.i(5), W = kp.i(6);
    i64 w = stream_width(dt, vec), M = N / w;
    const char *dn = dt == 0 ? (vec ? "float32x4" : "float32") : (vec ? "float64x2" : "float64");
    int ds = vec ? 16 : (dt == 0 ? 4 : 8);
    Out o(v);
    o.op((int)dt, 0, (u64)((L - 1) * w * M), (u64)((L - 1) * w * (M / 32)));
    static const char *nm[4] = {"in0", "in1", "in2", "in3"};
    Site st{};
    st.mem = GL; st.dtype = dn; st.dsize = ds;
    if (shape == 0) { st.nl = 1; st.l[0] = s; st.ng = 2; st.g[0] = 1; st.g[1] = 256 * s; }
    else { st.nl = 2; st.l[0] = 1; st.l[1] = W; st.ng = 2; st.g[0] = 16; st.g[1] = 16 * W; }
    st.wi = M; st.sg = M / 32; st.foot = M;
    for (int a = 0; a < L; a++) { st.tag = nm[a]; st.dir = LD; o.site(st); }
    st.tag = "out"; st.dir = ST; o.site(st);
    o.finish(0, M / 256);
    return PM_OK;
}

// Linear-id site of the 1-D, 256-wide kernels: index 256*gid0 + lid0.
Site lin_site(const char *tag, int dir, const char *dn, int ds, u64 T) {
    Site s{};
    s.tag = tag; s.mem = GL; s.dir = dir; s.dtype = dn; s.dsize = ds;
    s.nl = 1; s.l[0] = 1; s.ng = 1; s.g[0] = 256;
    s.wi = T; s.sg = T / 32; s.foot = T;
    return s;
}
// Local site with index lid0 + off (off fixed): footprint 256.
Site loc_site(const char *tag, int dir, u64 wi, u64 sg) {
    Site s{};
    s.tag = tag; s.mem = LO; s.dir = dir; s.dtype = "float32"; s.dsize = 4;
    s.nl = 1; s.l[0] = 1; s.ng = 1; s.g[0] = 0;
    s.wi = wi; s.sg = sg; s.foot = 256;
    return s;
}

pm_status counts_fma(const KP &kp, std::vector<pm_feature> &v) {
    i64 dt = kp.i(0), op = kp.i(1), F = kp.i(2), G = kp.i(3);
    const char *dn = dt == 0 ? "float32" : "float64";
    int ds = dt == 0 ? 4 : 8;
    u64 T = (u64)G * 256, S = (u64)G * 8;
    Out o(v);
    u64 adds = 32 + 31 + (op == 0 ? F : 0);
    o.op((int)dt, 0, T * adds, S * adds);
    if (op != 0) o.op((int)dt, (int)op, T * (u64)F, S * (u64)F);
    o.site(lin_site("seed", LD, dn, ds, T));
    o.site(lin_site("out", ST, dn, ds, T));
    o.finish(0, (u64)G);
    return PM_OK;
}

pm_status counts_smem(const KP &kp, std::vector<pm_feature> &v) {
    i64 R = kp.i(0), sync = kp.i(1), G = kp.i(2);
    u64 T = (u64)G * 256, S = (u64)G * 8, it = (u64)(R / 4);
    Out o(v);
    o.site(lin_site("in", LD, "float32", 4, T));
    o.site(loc_site("s_init", ST, T, S));
    o.site(loc_site("s_ldA", LD, T * it, S * it));
    o.site(loc_site("s_stB", ST, T * it, S * it));
    o.site(loc_site("s_ldB", LD, T * it, S * it));
    o.site(loc_site("s_stA", ST, T * it, S * it));
    o.site(loc_site("s_fin", LD, T, S));
    o.site(lin_site("out", ST, "float32", 4, T));
    o.finish(1 + (sync ? it : 0), (u64)G);
    return PM_OK;
}

// 2-D local shuffle: T x T work-group, local index T lid1 + lid0, all lanes
// active, ceil(T^2 / 32) sub-groups per group.
pm_status counts_smem2d(const KP &kp, std::vector<pm_feature> &v) {
    i64 R = kp.i(0), T = kp.i(1), G = kp.i(2);
    u64 W = (u64)(G * T * T), S = (u64)(G * ((T * T + 31) / 32)), it = (u64)(R / 4), TT = (u64)(T * T);
    Out o(v);
    auto gsite = [&](const char *tag, int dir) {
        Site s{};
        s.tag = tag; s.mem = GL; s.dir = dir; s.dtype = "float32"; s.dsize = 4;
        s.nl = 2; s.l[0] = 1; s.l[1] = T; s.ng = 1; s.g[0] = T * T;
        s.wi = W; s.sg = S; s.foot = W;
        return s;
    };
    auto lsite = [&](const char *tag, int dir, u64 reps, i64 loop) {
        Site s{};
        s.tag = tag; s.mem = LO; s.dir = dir; s.dtype = "float32"; s.dsize = 4;
        s.nl = 2; s.l[0] = 1; s.l[1] = T; s.ng = 1; s.g[0] = 0; s.loop = loop;
        s.wi = W * reps; s.sg = S * reps; s.foot = TT;
        return s;
    };
    o.site(gsite("in", LD));
    o.site(lsite("s_init", ST, 1, 0));
    o.site(lsite("s_ldA", LD, it, 0));
    o.site(lsite("s_stB", ST, it, 0));
    o.site(lsite("s_ldB", LD, it, 0));
    o.site(lsite("s_stA", ST, it, 0));
    o.site(lsite("s_fin", LD, 1, 0));
    o.site(gsite("out", ST));
    o.finish(1, (u64)G);
    return PM_OK;
}

pm_status counts_barrier(const KP &kp, std::vector<pm_feature> &v) {
    i64 B = kp.i(0), G = kp.i(1);
    u64 T = (u64)G * 256;
    Out o(v);
    o.site(lin_site("in", LD, "float32", 4, T));
    o.site(lin_site("out", ST, "float32", 4, T));
    o.finish((u64)B, (u64)G);
    return PM_OK;
}

pm_status counts_overlap(const KP &kp, std::vector<pm_feature> &v) {
    i64 m = kp.i(0), N = kp.i(1);
    u64 T = (u64)N, S = T / 32;
    Out o(v);
    o.site(lin_site("in", LD, "float32", 4, T));
    o.site(loc_site("s_st", ST, T * (u64)m, S * (u64)m));
    o.site(loc_site("s_ld", LD, T * (u64)m, S * (u64)m));
    o.site(lin_site("out", ST, "float32", 4, T));
    o.finish(0, T / 256);
    return PM_OK;
}

pm_status counts_empty(const KP &kp, std::vector<pm_feature> &v) {
    Out o(v);
    o.finish(0, (u64)kp.i(0));
    return PM_OK;
}

// ---------------------------------------------------------------- matmul
pm_status counts_mm(const KP &kp, std::vector<pm_feature> &v) {
    i64 n = kp.i(0);
    int var = kp.def->variant;
    u64 N2 = (u64)n * n, S2 = N2 / 32, K = (u64)(n / 16);
    Out o(v);
    auto gsite = [&](const char *tag, int dir, i64 l0, i64 l1, i64 g0, i64 g1, i64 loop, u64 wi, u64 sg) {
        Site s{};
        s.tag = tag; s.mem = GL; s.dir = dir; s.dtype = "float32"; s.dsize = 4;
        s.nl = 2; s.l[0] = l0; s.l[1] = l1; s.ng = 2; s.g[0] = g0; s.g[1] = g1; s.loop = loop;
        s.wi = wi; s.sg = sg; s.foot = N2;
        o.site(s);
    };
    auto lsite = [&](const char *tag, int dir, i64 l0, i64 l1, i64 loop, u64 wi, u64 sg) {
        Site s{};
        s.tag = tag; s.mem = LO; s.dir = dir; s.dtype = "float32"; s.dsize = 4;
        s.nl = 2; s.l[0] = l0; s.l[1] = l1; s.ng = 2; s.loop = loop;
        s.wi = wi; s.sg = sg; s.foot = 256;
        o.site(s);
    };
    const char *ta = var == 0 || var == 2 ? "mm-PF-a" : "mm-noPF-a";
    const char *tb = var == 0 || var == 3 ? "mm-PF-b" : "mm-noPF-b";
    switch (var) {
    case 0:  // PF: per k-tile: 2 fetches, 2 barriers, 16 madds
        o.op(0, 2, N2 * (u64)n, S2 * (u64)n);
        gsite(ta, LD, 1, n, 0, 16 * n, 16, N2 * K, S2 * K);
        lsite("a_fetch_st", ST, 1, 16, 0, N2 * K, S2 * K);
        gsite(tb, LD, 1, n, 16, 0, 16 * n, N2 * K, S2 * K);
        lsite("b_fetch_st", ST, 1, 16, 0, N2 * K, S2 * K);
        lsite("a_fetch_ld", LD, 0, 16, 1, N2 * (u64)n, S2 * (u64)n);
        lsite("b_fetch_ld", LD, 1, 0, 16, N2 * (u64)n, S2 * (u64)n);
        gsite("c", ST, 1, n, 16, 16 * n, 0, N2, S2);
        o.finish(2 * K, N2 / 256);
        break;
    case 1:  // noPF
        o.op(0, 2, N2 * (u64)n, S2 * (u64)n);
        gsite(ta, LD, 0, n, 0, 16 * n, 1, N2 * (u64)n, S2 * (u64)n);
        gsite(tb, LD, 1, 0, 16, 0, n, N2 * (u64)n, S2 * (u64)n);
        gsite("c", ST, 1, n, 16, 16 * n, 0, N2, S2);
        o.finish(0, N2 / 256);
        break;
    default: {  // work-removed twins: tgt += x per kept load, then tgt_dest
        u64 per = (var == 2 || var == 3) ? K : (u64)n;
        o.op(0, 0, N2 * per, S2 * per);
        if (var == 2) gsite(ta, LD, 1, n, 0, 16 * n, 16, N2 * K, S2 * K);
        if (var == 3) gsite(tb, LD, 1, n, 16, 0, 16 * n, N2 * K, S2 * K);
        if (var == 4) gsite(ta, LD, 0, n, 0, 16 * n, 1, N2 * (u64)n, S2 * (u64)n);
        if (var == 5) gsite(tb, LD, 1, 0, 16, 0, n, N2 * (u64)n, S2 * (u64)n);
        gsite("tgt_dest", ST, 1, n, 16, 16 * n, 0, N2, S2);
        o.finish(0, N2 / 256);
    }
    }
    return PM_OK;
}

// ---------------------------------------------------------------- DG
// k = L0*gid0 + lid0, i = L1*gid1 + lid1, guard i < Np.  A sub-group holds
// r = 32/L0 whole rows (lid1 values); rows never straddle work-groups since
// L1 is a multiple of r, so the number of sub-groups with an active first
// row, per gid0, is ceil(Np / r).
pm_status counts_dg(const KP &kp, std::vector<pm_feature> &v) {
    i64 Np = kp.i(0), Nel = kp.i(1), L0 = kp.i(2), L1 = kp.i(3);
    int var = kp.def->variant;
    i64 G0 = Nel / L0, G1 = cdiv(Np, L1), r = 32 / L0, nj = cdiv(Np, L0);
    u64 SGa = (u64)(G0 * cdiv(Np, r));          // active sub-groups
    u64 WIa = (u64)(Nel * Np);                   // active work-items
    u64 Np2 = (u64)(Np * Np);
    u64 WIall = (u64)(G0 * G1 * L0 * L1), SGall = (u64)(G0 * G1 * (L0 * L1 / 32));
    char t_nu[32], t_ndm[32], t_pu[32], t_pdm[32], t_res[32], t_uu[32], t_tu[32], t_tres[32];
    snprintf(t_uu, sizeof t_uu, "dg-uPF-u-%dx%d", (int)L0, (int)L1);
    snprintf(t_tu, sizeof t_tu, "dg-dmPFT-u-%dx%d", (int)L0, (int)L1);
    snprintf(t_tres, sizeof t_tres, "dg-dmPFT-res-%dx%d", (int)L0, (int)L1);
    snprintf(t_nu, sizeof t_nu, "dg-noPF-u-%dx%d", (int)L0, (int)L1);
    snprintf(t_ndm, sizeof t_ndm, "dg-noPF-dm-%dx%d", (int)L0, (int)L1);
    snprintf(t_pu, sizeof t_pu, "dg-dmPF-u-%dx%d", (int)L0, (int)L1);
    snprintf(t_pdm, sizeof t_pdm, "dg-dmPF-dm-%dx%d", (int)L0, (int)L1);
    snprintf(t_res, sizeof t_res, "dg-res-%dx%d", (int)L0, (int)L1);
    Out o(v);
    auto site = [&](const char *tag, int mem, int dir, i64 l0, i64 l1, i64 g0, i64 g1, i64 loop, u64 wi, u64 sg,
                    u64 foot) {
        Site s{};
        s.tag = tag; s.mem = mem; s.dir = dir; s.dtype = "float32"; s.dsize = 4;
        s.nl = 2; s.l[0] = l0; s.l[1] = l1; s.ng = 2; s.g[0] = g0; s.g[1] = g1; s.loop = loop;
        s.wi = wi; s.sg = sg; s.foot = foot;
        o.site(s);
    };
    const u64 inner = 3 * (u64)Np;  // (m, j) instances per active work-item
    // u[Np*k + j], D[Np^2 m + Np i + j], res[Nel Np m + Np k + i]
    auto u_site = [&](const char *tag) {
        site(tag, GL, LD, Np, 0, L0 * Np, 0, 1, WIa * inner, SGa * inner, (u64)(Nel * Np));
    };
    auto d_site = [&](const char *tag) {
        site(tag, GL, LD, 0, Np, 0, L1 * Np, 1, WIa * inner, SGa * inner, 3 * Np2);
    };
    auto res_site = [&]() {
        site(t_res, GL, ST, Np, 1, L0 * Np, L1, Nel * Np, WIa * 3, SGa * 3, (u64)(3 * Nel * Np));
    };
    auto dest_site = [&]() {
        site("tgt_dest", GL, ST, 1, Nel, L0, L1 * Nel, 0, WIall, SGall, WIall);
    };
    // dmPF D fetch: guard i < Np and L0*jo + lid0 < Np; per (m, jo) the active
    // columns over all jo total Np, so work-items 3 G0 Np^2; every active
    // sub-group has an active lane for every jo.
    u64 fWI = 3 * (u64)G0 * Np2, fSG = 3 * (u64)nj * SGa;
    u64 tileFoot = (u64)(std::min(L1, Np) * std::min(L0, Np));
    switch (var) {
    case 0:
        o.op(0, 2, WIa * inner, SGa * inner);
        d_site(t_ndm);
        u_site(t_nu);
        res_site();
        o.finish(0, (u64)(G0 * G1));
        break;
    case 1:
        o.op(0, 2, WIa * inner, SGa * inner);
        site(t_pdm, GL, LD, 1, Np, 0, L1 * Np, L0, fWI, fSG, 3 * Np2);
        site("dm_fetch_st", LO, ST, 1, L0, 0, 0, 0, fWI, fSG, tileFoot);
        site("dm_fetch_ld", LO, LD, 0, L0, 0, 0, 1, WIa * inner, SGa * inner, tileFoot);
        site(t_pu, GL, LD, Np, 0, L0 * Np, 0, 1, WIa * inner, SGa * inner, (u64)(Nel * Np));
        res_site();
        o.finish(6 * (u64)nj, (u64)(G0 * G1));
        break;
    case 2: case 3:
        o.op(0, 0, WIa * inner, SGa * inner);
        if (var == 2) u_site(t_nu);
        else d_site(t_ndm);
        dest_site();
        o.finish(0, (u64)(G0 * G1));
        break;
    case 4:
        o.op(0, 0, WIa * inner, SGa * inner);
        site(t_pu, GL, LD, Np, 0, L0 * Np, 0, 1, WIa * inner, SGa * inner, (u64)(Nel * Np));
        dest_site();
        o.finish(0, (u64)(G0 * G1));
        break;
    case 5:
        o.op(0, 0, fWI, fSG);
        site(t_pdm, GL, LD, 1, Np, 0, L1 * Np, L0, fWI, fSG, 3 * Np2);
        dest_site();
        o.finish(0, (u64)(G0 * G1));
        break;
    case 6:
        res_site();
        o.finish(0, (u64)(G0 * G1));
        break;
    case 7: case 9: {
        // uPF (L0 == L1): per j tile every work-item (any row) with
        // L1 jo + lid0 < Np fetches u[Np (L0 gid0 + lid1) + L1 jo + lid0];
        // summed over the tiles that is L1 Np per group, and every sub-group
        // has an active lane (lid0 = 0) in every tile.
        i64 njl = cdiv(Np, L1);
        u64 uWI = (u64)(G0 * G1 * L1 * Np), uSG = (u64)(G0 * G1 * (L0 * L1 / 32) * njl);
        u64 ufoot = (u64)(L0 * std::min(L1, Np));
        if (var == 7) {
            o.op(0, 2, WIa * inner, SGa * inner);
            site(t_uu, GL, LD, 1, Np, L0 * Np, 0, L1, uWI, uSG, (u64)(Nel * Np));
            site("u_fetch_st", LO, ST, 1, L1 + 1, 0, 0, 0, uWI, uSG, ufoot);
            site("u_fetch_ld", LO, LD, L1 + 1, 0, 0, 0, 1, WIa * (u64)Np, SGa * (u64)Np, ufoot);
            site(t_ndm, GL, LD, 0, Np, 0, L1 * Np, Np * Np, WIa * inner, SGa * inner, 3 * Np2);
            res_site();
            o.finish(2 * (u64)njl, (u64)(G0 * G1));
        } else {
            o.op(0, 0, uWI, uSG);
            site(t_uu, GL, LD, 1, Np, L0 * Np, 0, L1, uWI, uSG, (u64)(Nel * Np));
            dest_site();
            o.finish(0, (u64)(G0 * G1));
        }
        break;
    }
    case 8:
        // dmPF-T: dmPF on uT[j, k] = Nel j + k and resT[m, i, k] = Nel Np m + Nel i + k
        o.op(0, 2, WIa * inner, SGa * inner);
        site(t_pdm, GL, LD, 1, Np, 0, L1 * Np, L0, fWI, fSG, 3 * Np2);
        site("dm_fetch_st", LO, ST, 1, L0, 0, 0, 0, fWI, fSG, tileFoot);
        site("dm_fetch_ld", LO, LD, 0, L0, 0, 0, 1, WIa * inner, SGa * inner, tileFoot);
        site(t_tu, GL, LD, 1, 0, L0, 0, Nel, WIa * inner, SGa * inner, (u64)(Nel * Np));
        site(t_tres, GL, ST, 1, Nel, L0, L1 * Nel, Nel * Np, WIa * 3, SGa * 3, (u64)(3 * Nel * Np));
        o.finish(6 * (u64)nj, (u64)(G0 * G1));
        break;
    case 10:
        o.op(0, 0, WIa * inner, SGa * inner);
        site(t_tu, GL, LD, 1, 0, L0, 0, Nel, WIa * inner, SGa * inner, (u64)(Nel * Np));
        dest_site();
        o.finish(0, (u64)(G0 * G1));
        break;
    case 11:
        site(t_tres, GL, ST, 1, Nel, L0, L1 * Nel, Nel * Np, WIa * 3, SGa * 3, (u64)(3 * Nel * Np));
        o.finish(0, (u64)(G0 * G1));
        break;
    }
    return PM_OK;
}

// ---------------------------------------------------------------- stencil
pm_status counts_fd(const KP &kp, std::vector<pm_feature> &v) {
    i64 n = kp.i(0), W = n + 2;
    int var = kp.def->variant;
    Out o(v);
    auto site = [&](const char *tag, int mem, int dir, i64 l0, i64 l1, i64 g0, i64 g1, u64 wi, u64 sg, u64 foot) {
        Site s{};
        s.tag = tag; s.mem = mem; s.dir = dir; s.dtype = "float32"; s.dsize = 4;
        s.nl = 2; s.l[0] = l0; s.l[1] = l1; s.ng = 2; s.g[0] = g0; s.g[1] = g1;
        s.wi = wi; s.sg = sg; s.foot = foot;
        o.site(s);
    };
    u64 N2 = (u64)(n * n);
    if (var >= 6) {
        // 18x18 work-group (tid = lid0 + 18 lid1), tile origin 16 gid; the
        // active lanes of a statement form a rectangle per group, whose extent
        // depends only on whether the group is the last one along each axis.
        const i64 T = 18, S = 16, G = cdiv(n, S);
        auto sg_rect = [&](i64 x0, i64 x1, i64 y0, i64 y1) {
            u64 c = 0;
            for (i64 q = 0; q * 32 < T * T; q++) {
                bool any = false;
                for (i64 t = 32 * q; t < std::min(32 * q + 32, T * T) && !any; t++)
                    any = t % T >= x0 && t % T < x1 && t / T >= y0 && t / T < y1;
                c += any;
            }
            return c;
        };
        // per-axis extents: fetch rows min(T, W - S g), computing rows min(S, n - S g)
        i64 fe[2] = {std::min(T, W), std::min(T, W - S * (G - 1))};
        i64 ce[2] = {std::min(S, n), std::min(S, n - S * (G - 1))};
        u64 cnt[2] = {(u64)(G - 1), 1};   // groups 0..G-2 are full, group G-1 is the last
        u64 fWI = 0, fSG = 0, cSG = 0;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                u64 m = cnt[a] * cnt[b];
                if (!m) continue;
                fWI += m * (u64)(fe[a] * fe[b]);
                fSG += m * sg_rect(0, fe[a], 0, fe[b]);
                cSG += m * sg_rect(1, 1 + ce[a], 1, 1 + ce[b]);
            }
        if (G == 1) {   // the only group is the last one: recount without the "full" class
            fWI = (u64)(fe[1] * fe[1]);
            fSG = sg_rect(0, fe[1], 0, fe[1]);
            cSG = sg_rect(1, 1 + ce[1], 1, 1 + ce[1]);
        }
        u64 tf = (u64)(std::min(T, W) * std::min(T, W)), cf = (u64)(std::min(S, n) * std::min(S, n));
        if (var == 6) {
            o.op(0, 0, 3 * N2, 3 * cSG);
            o.op(0, 1, N2, cSG);
            o.op(0, 2, N2, cSG);
            site("fd-tile18-u", GL, LD, 1, W, S, S * W, fWI, fSG, (u64)(W * W));
            site("u_fetch_st", LO, ST, 1, T, 0, 0, fWI, fSG, tf);
            static const char *nm[5] = {"u_fetch_c", "u_fetch_n", "u_fetch_s", "u_fetch_w", "u_fetch_e"};
            for (int k = 0; k < 5; k++) site(nm[k], LO, LD, 1, T, 0, 0, N2, cSG, cf);
            site("fd-tile18-res", GL, ST, 1, n, S, S * n, N2, cSG, N2);
            o.finish(1, (u64)(G * G));
        } else if (var == 7) {
            o.op(0, 0, fWI, fSG);
            site("fd-tile18-u", GL, LD, 1, W, S, S * W, fWI, fSG, (u64)(W * W));
            u64 all = (u64)(T * T * G * G), allSG = (u64)(cdiv(T * T, 32) * G * G);
            site("tgt_dest", GL, ST, 1, T * G, T, T * T * G, all, allSG, all);
            o.finish(0, (u64)(G * G));
        } else {
            site("fd-tile18-res", GL, ST, 1, n, S, S * n, N2, cSG, N2);
            o.finish(0, (u64)(G * G));
        }
    } else if (var == 0 || var == 2 || var == 3) {
        // 16x16 work-group, tile origin 14*gid; a sub-group is rows {2q, 2q+1}.
        i64 G = cdiv(n, 14);
        u64 S = 0, Qf = 0, Qc = 0;
        for (i64 g = 0; g < G; g++) {
            S += (u64)std::min<i64>(16, W - 14 * g);             // fetching rows (or columns) of tile g
            Qf += (u64)std::min<i64>(8, cdiv(W - 14 * g, 2));    // sub-groups with a fetching first row
            Qc += (u64)(std::min<i64>(14, n - 14 * g) / 2 + 1);  // sub-groups with a computing row
        }
        u64 fWI = S * S, fSG = (u64)G * Qf, cSG = (u64)G * Qc;
        u64 tf = (u64)(std::min<i64>(16, W) * std::min<i64>(16, W));
        u64 cf = (u64)(std::min<i64>(14, n) * std::min<i64>(14, n));
        if (var == 0) {
            o.op(0, 0, 3 * N2, 3 * cSG);
            o.op(0, 1, N2, cSG);
            o.op(0, 2, N2, cSG);
            site("fd-tile-u", GL, LD, 1, W, 14, 14 * W, fWI, fSG, (u64)(W * W));
            site("u_fetch_st", LO, ST, 1, 16, 0, 0, fWI, fSG, tf);
            static const char *nm[5] = {"u_fetch_c", "u_fetch_n", "u_fetch_s", "u_fetch_w", "u_fetch_e"};
            for (int k = 0; k < 5; k++) site(nm[k], LO, LD, 1, 16, 0, 0, N2, cSG, cf);
            site("fd-tile-res", GL, ST, 1, n, 14, 14 * n, N2, cSG, N2);
            o.finish(1, (u64)(G * G));
        } else if (var == 2) {
            o.op(0, 0, fWI, fSG);
            site("fd-tile-u", GL, LD, 1, W, 14, 14 * W, fWI, fSG, (u64)(W * W));
            u64 all = (u64)(256 * G * G);
            site("tgt_dest", GL, ST, 1, 16 * G, 16, 256 * G, all, all / 32, all);
            o.finish(0, (u64)(G * G));
        } else {
            site("fd-tile-res", GL, ST, 1, n, 14, 14 * n, N2, cSG, N2);
            o.finish(0, (u64)(G * G));
        }
    } else {
        i64 G = cdiv(n, 16);
        u64 Q = 0;
        for (i64 g = 0; g < G; g++) Q += (u64)std::min<i64>(8, cdiv(n - 16 * g, 2));
        u64 cSG = (u64)G * Q;
        static const char *nm[5] = {"u_c", "u_n", "u_s", "u_w", "u_e"};
        if (var == 1) {
            o.op(0, 0, 3 * N2, 3 * cSG);
            o.op(0, 1, N2, cSG);
            o.op(0, 2, N2, cSG);
            for (int k = 0; k < 5; k++) site(nm[k], GL, LD, 1, W, 16, 16 * W, N2, cSG, N2);
            site("res", GL, ST, 1, n, 16, 16 * n, N2, cSG, N2);
        } else if (var == 4) {
            o.op(0, 0, 5 * N2, 5 * cSG);
            for (int k = 0; k < 5; k++) site(nm[k], GL, LD, 1, W, 16, 16 * W, N2, cSG, N2);
            u64 all = (u64)(256 * G * G);
            site("tgt_dest", GL, ST, 1, 16 * G, 16, 256 * G, all, all / 32, all);
        } else {
            site("res", GL, ST, 1, n, 16, 16 * n, N2, cSG, N2);
        }
        o.finish(0, (u64)(G * G));
    }
    return PM_OK;
}

// ---------------------------------------------------------------- SIMT matmul family
// Work-group (BN/8) x (BM/8), 8x8 outputs per work-item, k tiles of BK; see
// pm_tiles.cu for the loop nest.  Vector (float32x4) units for global memory.
pm_status counts_simt(const KP &kp, std::vector<pm_feature> &v) {
    i64 n = kp.i(0), BM = kp.i(1), BN = kp.i(2), BK = kp.i(3);
    i64 L0 = BN / 8, L1 = BM / 8, T = L0 * L1, S = T / 32, KC = BK / 4, NC = BN / 4;
    i64 G = (n / BN) * (n / BM), K = n / BK, n4 = n / 4;
    i64 qa = cdiv(KC, L0);
    u64 aWI = (u64)(G * K * BM * KC), aSG = (u64)(G * S * K * 8 * qa);
    // B tile rows lid1 + L1 r < BK: a sub-group's first row a decides activity
    i64 bsg = 0;
    for (i64 sg = 0; sg < S; sg++) {
        i64 a = L0 >= 32 ? (32 * sg) / L0 : (32 * sg) / L0;
        bsg += 2 * cdiv(BK - a, L1);
    }
    u64 bWI = (u64)(G * K * BK * NC), bSG = (u64)(G * K * bsg);
    Out o(v);
    o.op(0, 2, (u64)(G * T * K * BK * 64), (u64)(G * S * K * BK * 64));
    auto site = [&](const char *tag, int mem, int dir, const char *dt, int ds, i64 l0, i64 l1, i64 g0, i64 g1,
                    i64 loop, u64 wi, u64 sg, u64 foot) {
        Site x{};
        x.tag = tag; x.mem = mem; x.dir = dir; x.dtype = dt; x.dsize = ds;
        x.nl = 2; x.l[0] = l0; x.l[1] = l1; x.ng = 2; x.g[0] = g0; x.g[1] = g1; x.loop = loop;
        x.wi = wi; x.sg = sg; x.foot = foot;
        o.site(x);
    };
    const u64 full = (u64)(n * n / 4);
    site("simt-a", GL, LD, "float32x4", 16, 1, n4, 0, BM * n4, L0, aWI, aSG, full);
    static const char *ast[4] = {"As_st0", "As_st1", "As_st2", "As_st3"};
    const i64 BMP = BM + 4;   // padded row of the transposed A tile
    for (int j = 0; j < 4; j++) site(ast[j], LO, ST, "float32", 4, 4 * BMP, 1, 0, 0, 4 * L0 * BMP, aWI, aSG, (u64)(BM * KC));
    site("simt-b", GL, LD, "float32x4", 16, 1, n4, NC, 0, L0, bWI, bSG, full);
    site("Bs_st", LO, ST, "float32x4", 16, 1, NC, 0, 0, L0, bWI, bSG, (u64)(BK * NC));
    const u64 cWI = (u64)(G * T * K * BK), cSG = (u64)(G * S * K * BK);
    site("As_ld0", LO, LD, "float32x4", 16, 0, 2, 0, 0, BMP / 4, cWI, cSG, (u64)(BK * L1));
    site("As_ld1", LO, LD, "float32x4", 16, 0, 2, 0, 0, BMP / 4, cWI, cSG, (u64)(BK * L1));
    site("Bs_ld0", LO, LD, "float32x4", 16, 1, 0, 0, 0, NC, cWI, cSG, (u64)(BK * L0));
    site("Bs_ld1", LO, LD, "float32x4", 16, 1, 0, 0, 0, NC, cWI, cSG, (u64)(BK * L0));
    site("simt-c", GL, ST, "float32x4", 16, 1, 2 * n, NC, BM * n4, L0, (u64)(G * T * 16), (u64)(G * S * 16), full);
    o.finish((u64)(2 * K), (u64)G);
    return PM_OK;
}

// ---------------------------------------------------------------- tensor-core matmul
// R-thread work-group per R x 256 tile of C (R = 128 for mm_tc, 256 for
// mm_tc256); per 64-wide k tile the elected thread 0 copies an Rx64 box of A
// and a 256x64 box of Bt (counted element by element, uniform, hence per
// sub-group) and thread 32 issues R/32 128x256x16 multiply-add instructions
// (R/128 row halves x 4 k slices); every work-item stores 64 16-byte vectors
// of its C row; three barriers.
pm_status counts_tc(const KP &kp, std::vector<pm_feature> &v) {
    i64 n = kp.i(0), R = kp.def->variant ? 256 : 128;
    u64 G = (u64)((n / 256) * (n / R)), KT = (u64)(n / 64);
    u64 nn = (u64)(n * n);
    Out o(v);
    auto site = [&](const char *tag, int dir, const char *dt, int ds, int nl, i64 l0, i64 g0, i64 g1, i64 loop, u64 wi,
                    u64 sg, u64 foot) {
        Site x{};
        x.tag = tag; x.mem = GL; x.dir = dir; x.dtype = dt; x.dsize = ds;
        x.nl = nl; x.l[0] = l0; x.ng = 2; x.g[0] = g0; x.g[1] = g1; x.loop = loop;
        x.wi = wi; x.sg = sg; x.foot = foot;
        o.site(x);
    };
    const u64 ma = G * KT * (u64)R * 64, mb = G * KT * 256 * 64, mm = G * KT * (u64)(R / 32);
    site("tc-a", LD, "bfloat16", 2, 1, 0, 0, R * n, 1, ma, ma, nn);
    site("tc-b", LD, "bfloat16", 2, 1, 0, 256 * n, 0, 1, mb, mb, nn);
    site("tc-c", ST, "float32x4", 16, 1, n / 4, 64, R * n / 4, 1, G * (u64)R * 64, G * (u64)(R / 32) * 64, nn / 4);
    pm_feature f = op_rec("bfloat16", "madd", mm * 128 * 256 * 16, mm * 128 * 256 * 16);
    v.push_back(f);
    for (auto &x : o.sites) v.push_back(x);
    v.push_back(simple(PM_FEAT_SYNC, PM_GRAN_WI, 3));
    v.push_back(simple(PM_FEAT_GROUPS, PM_GRAN_WG, G));
    v.push_back(simple(PM_FEAT_LAUNCH, PM_GRAN_K, 1));
    return PM_OK;
}

// ---------------------------------------------------------------- DG on the tensor cores
// Grid (G, P) of 320-thread work-groups, 352 with A = 1 (G = 3 / MS m-groups: MS = 3 m per
// work-group for Np <= 40, and for Np <= 64 with A = 0; P persistent
// work-groups per m-group, the default resolved as the launch resolves it);
// work-group (g, p) serves the tiles t = p, p + P, ... of 128 elements.
//   threads i < NP8, per m of the group (MS of them) and chunk ac < 8 KA of
//   the operator row: loads D[m, i, 4 ac + x] (i, 4 ac + x < Np), 4 adds
//   (the head/remainder split), two 16-byte shared stores (head, remainder);
//   threads below NR - MS NP8: two zero stores per chunk of the padding rows;
//   one barrier;
//   per tile and atom a (chunks c < CN(a) = 2 min(4, KS - 4a)):
//     Np % 4 == 0: thread 256 copies the in-range part of the 128 x 32 box
//       (counted per element, uniform); converter thread r = tid - 128 loads
//       chunk c of its row from the staged atom (16-byte shared load);
//     else, A = 1: thread 256 copies the tile's rows x Np elements (one bulk
//       copy per tile, counted per element, uniform); converter thread r
//       loads the row's four elements of chunk c from it (4-byte shared
//       loads, k = 128 t + r < Nel, j < Np);
//     else, A = 0: converter thread r loads the row's four elements of chunk
//       c from global memory (k = 128 t + r < Nel, j < Np);
//     converter: 4 adds per chunk; with A = 0 two 16-byte shared stores
//       (head, remainder); with A = 1 the chunk goes to tensor memory;
//     thread 288 (A = 1: 288 and 320 on alternate tiles): per k step 3 MMAs
//       of 128 x NR x 8 TF32 multiply-adds;
//   per tile, epilogue threads tid < 128, per m: the store of the thread's
//   row to the staging buffer (Np / 4 16-byte stores, or Np 4-byte stores
//   when Np % 4 != 0), and thread 0 copies the block's rows x Np elements to
//   res (counted per element, uniform);
//   two barriers at the end.  The epilogue warps' named barriers among
//   themselves (128 of the threads) are not work-group barriers and are
//   not counted: every thread passes the same three work-group barriers.
// Shared-memory sites are given by their logical position (row, chunk) in
// one ring stage or staging buffer: the swizzle permutes 16-byte chunks
// within a 128-byte row and the ring rotates whole stages, which changes
// neither counts nor footprints.
pm_status counts_dgc(const KP &kp, std::vector<pm_feature> &v) {
    const i64 Np = kp.i(0), Nel = kp.i(1);
    const int A = dgc_resolve_a((int)Np, (int)kp.i(3));
    const i64 P = dgc_resolve_p((int)Np, Nel, A, (int)kp.i(2));
    const i64 MS = dgc_geometry((int)Np, A).ms, G = 3 / MS, NP8 = (Np + 7) / 8 * 8, NR = (MS * NP8 + 15) / 16 * 16;
    const i64 KA = cdiv(Np, 32), KS = cdiv(Np, 8), CN0 = 2 * std::min<i64>(4, KS), PAD = NR - MS * NP8;
    const bool tma = Np % 4 == 0;
    const i64 T = cdiv(Nel, 128), Tf = Nel / 128, rl = Nel % 128;
    const u64 sum_sg_rows = (u64)(4 * Tf + (rl ? cdiv(rl, 32) : 0));   // sum over tiles of ceil(rows / 32)
    const u64 GP = (u64)(G * P), GT = (u64)(G * T), uNp = (u64)Np;
    Out o(v);
    auto site = [&](const char *tag, int mem, int dir, const char *dt, int ds, i64 l0, i64 g0, i64 g1, u64 wi, u64 sg,
                    u64 foot) {
        Site x{};
        x.tag = tag; x.mem = mem; x.dir = dir; x.dtype = dt; x.dsize = ds;
        x.nl = 1; x.l[0] = l0; x.ng = 2; x.g[0] = g0; x.g[1] = g1; x.loop = 1;
        x.wi = wi; x.sg = sg; x.foot = foot;
        o.site(x);
    };
    // operator staging
    site("dgc-D", GL, LD, "float32", 4, Np, MS == 1 ? Np * Np : 0, 0, GP * (u64)MS * uNp * uNp,
         GP * (u64)MS * uNp * (u64)cdiv(Np, 32), (u64)(3 * Np * Np));
    const u64 bst = (u64)(8 * KA) * (u64)NR * GP;
    const u64 bsg = (u64)(8 * KA) * GP * (u64)(MS * cdiv(NP8, 32) + cdiv(PAD, 32));
    site("dgc-Bh", LO, ST, "float32x4", 16, 8 * KA, 0, 0, bst, bsg, (u64)(NR * 8 * KA));
    site("dgc-Bl", LO, ST, "float32x4", 16, 8 * KA, 0, 0, bst, bsg, (u64)(NR * 8 * KA));
    o.op(0, 0, 4 * GP * (u64)(MS * NP8 * 8 * KA), 4 * GP * (u64)(MS * cdiv(NP8, 32) * 8 * KA));
    // u operand
    const u64 uel = (u64)(G * Nel) * uNp;
    const bool bulk = !tma && A == 1;   // A = 1, Np % 4 != 0: one bulk copy of the tile's rows
    if (tma || bulk) site("dgc-u", GL, LD, "float32", 4, 0, 0, 128 * Np, uel, uel, (u64)(Nel * Np));
    else site("dgc-u", GL, LD, "float32", 4, Np, 0, 128 * Np, uel, (u64)G * uNp * sum_sg_rows, (u64)(Nel * Np));
    if (bulk)
        site("dgc-R", LO, LD, "float32", 4, Np, 0, 0, uel, (u64)G * uNp * sum_sg_rows,
             (u64)(std::min<i64>(128, Nel) * Np));
    const u64 cwi = GT * (u64)(2 * KS) * 128, csg = GT * (u64)(2 * KS) * 4;
    if (tma) site("dgc-Ur", LO, LD, "float32x4", 16, 8, 0, 0, cwi, csg, (u64)(128 * CN0));
    if (A == 0) {
        site("dgc-Uh", LO, ST, "float32x4", 16, 8, 0, 0, cwi, csg, (u64)(128 * CN0));
        site("dgc-Ul", LO, ST, "float32x4", 16, 8, 0, 0, cwi, csg, (u64)(128 * CN0));
    }
    o.op(0, 0, 4 * cwi, 4 * csg);
    // epilogue
    if (Np % 4 == 0)
        site("dgc-O", LO, ST, "float32x4", 16, Np / 4, 0, 0, GT * (u64)MS * 128 * (uNp / 4),
             GT * (u64)MS * 4 * (uNp / 4), (u64)(128 * Np / 4));
    else
        site("dgc-O", LO, ST, "float32", 4, Np, 0, 0, GT * (u64)MS * 128 * uNp, GT * (u64)MS * 4 * uNp,
             (u64)(128 * Np));
    const u64 rel = (u64)(3 * Nel) * uNp;
    site("dgc-res", GL, ST, "float32", 4, 0, MS == 1 ? Nel * Np : 0, 128 * Np, rel, rel, rel);
    const u64 mm = GT * (u64)KS * 3 * 128 * (u64)NR * 8;
    v.push_back(op_rec("tfloat32", "madd", mm, mm));
    o.finish(3, GP);
    return PM_OK;
}

// ---------------------------------------------------------------- stencil tile family
// Work-group (BX/4) x BY, input pitch P = n + 4; work-item (0,0) copies the
// (BY+2) x (BX+4) box element by element (uniform: per sub-group); every
// work-item loads 14 shared values, computes 4 outputs, stores one vector.
pm_status counts_fdb(const KP &kp, std::vector<pm_feature> &v) {
    i64 n = kp.i(0), BX = kp.i(1), BY = kp.i(2), V = kp.i(5), P = n + 4;
    i64 L0 = BX / V, L1 = BY, T = L0 * L1, G = (n / BX) * (n / BY), TW = BX + 4;
    u64 SGw = (u64)((T + 31) / 32);   // sub-groups per work-group
    Out o(v);
    const u64 WI = (u64)(G * T), SG = (u64)G * SGw;
    o.op(0, 0, 3 * V * WI, 3 * V * SG);
    o.op(0, 1, V * WI, V * SG);
    o.op(0, 2, V * WI, V * SG);
    auto site = [&](const char *tag, int mem, int dir, const char *dt, int ds, i64 l0, i64 l1, i64 g0, i64 g1,
                    i64 loop, u64 wi, u64 sg, u64 foot) {
        Site x{};
        x.tag = tag; x.mem = mem; x.dir = dir; x.dtype = dt; x.dsize = ds;
        x.nl = 2; x.l[0] = l0; x.l[1] = l1; x.ng = 2; x.g[0] = g0; x.g[1] = g1; x.loop = loop;
        x.wi = wi; x.sg = sg; x.foot = foot;
        o.site(x);
    };
    const u64 box = (u64)((BY + 2) * (BX + 4)) * (u64)G;
    site("fdb-u", GL, LD, "float32", 4, 0, 0, BX, BY * P, 1, box, box, (u64)((n + 2) * P));
    // shared loads: centre row columns V lid0 + 0..V+1, north and south rows V lid0 + 1..V
    site("t_c", LO, LD, "float32", 4, V, TW, 0, 0, 1, WI * (V + 2), SG * (V + 2), (u64)(BY * (BX + 2)));
    site("t_n", LO, LD, "float32", 4, V, TW, 0, 0, 1, WI * V, SG * V, (u64)(BY * BX));
    site("t_s", LO, LD, "float32", 4, V, TW, 0, 0, 1, WI * V, SG * V, (u64)(BY * BX));
    site("fdb-res", GL, ST, "float32x4", 16, V / 4, n / 4, BX / 4, BY * n / 4, 1, WI * (V / 4), SG * (V / 4),
         (u64)(n * n / 4));
    o.finish(1, (u64)G);
    return PM_OK;
}

// ---------------------------------------------------------------- DG tile
// XL x 16 work-group per (m, 128 elements), grid (3, ceil(Nel / 128)):
// NB = ceil(Np / 16) columns per work-item, XL = ceil(Np / NB) x-lanes, node
// rows padded to NPP = XL NB, j in Q = ceil(Np / 2) pairs (8-byte vectors),
// Dt row pitch PD (PD >= 2 Q, PD % 32 == 2).  Work-item (x, y): D staging for
// row i = y + 16 ib (ib < ceil(NPP / 16)) and pair q = x + XL qb < Q -- a
// vector load of D[m, i, 2q ..] when Np is even (else the j < Np elements one
// by one) for i < Np, a vector store to Dt[i][q] for i < NPP; work-item
// (0, 0) copies the u tile (one bulk copy, counted per element); when Np is
// odd the 128 rows are re-laid out with pitch 2 Q (element loads, vector
// stores) behind a second barrier; then per pair: 8 vector loads of
// Us[y + 16 a][q], NB of Dt[x + XL b][q], 2 x 8 x NB madds (running sums
// over the even and the odd j); per output one add of its two sums, then
// the store res[m, k0 + y + 16 a, x + XL b] (k < Nel, i < Np).  A sub-group is 32
// consecutive linear ids t = x + XL y; its count for a statement instance is
// taken over the work-group's lanes directly (at most 256 of them).
pm_status counts_dgt(const KP &kp, std::vector<pm_feature> &v) {
    const i64 Np = kp.i(0), Nel = kp.i(1), NB = cdiv(Np, 16), XL = cdiv(Np, NB), NPP = XL * NB;
    const i64 Q = cdiv(Np, 2), QB = cdiv(Q, XL), RB = cdiv(NPP, 16), NT = 16 * XL, NW = cdiv(NT, 32);
    i64 PD = 2 * Q;
    while (PD % 32 != 2) PD++;
    const bool even = Np % 2 == 0;
    const i64 T = cdiv(Nel, 128), Tfull = Nel / 128, rlast = Nel % 128, G = 3 * T;
    const u64 uG = (u64)G, uNp = (u64)Np, uQ = (u64)Q, uNB = (u64)NB;
    // active sub-groups of one work-group for a lane predicate pred(x, y)
    auto sg = [&](auto pred) {
        u64 n = 0;
        for (i64 w = 0; w < NW; w++) {
            bool any = false;
            for (i64 t = 32 * w; t < std::min(32 * w + 32, NT) && !any; t++) any = pred(t % XL, t / XL);
            n += any;
        }
        return n;
    };
    u64 sg_D = 0, sg_Dt = 0, sg_R = 0, sg_Ur = 0, sg_res_full = 0, sg_res_last = 0;
    for (i64 ib = 0; ib < RB; ib++)
        for (i64 qb = 0; qb < QB; qb++) {
            auto in = [&](i64 x, i64 y) { return x + XL * qb < Q && y + 16 * ib < Np; };
            if (even) {
                sg_D += sg(in);
            } else {
                for (i64 e = 0; e < 2; e++)
                    sg_D += sg([&](i64 x, i64 y) { return in(x, y) && 2 * (x + XL * qb) + e < Np; });
            }
            sg_Dt += sg([&](i64 x, i64 y) { return x + XL * qb < Q && y + 16 * ib < NPP; });
        }
    for (i64 qb = 0; qb < QB; qb++) {
        for (i64 e = 0; e < 2; e++)
            sg_R += 8 * sg([&](i64 x, i64) { return x + XL * qb < Q && 2 * (x + XL * qb) + e < Np; });
        sg_Ur += 8 * sg([&](i64 x, i64) { return x + XL * qb < Q; });
    }
    for (i64 b = 0; b < NB; b++)
        for (i64 a = 0; a < 8; a++) {
            sg_res_full += sg([&](i64 x, i64) { return x + XL * b < Np; });
            if (rlast) sg_res_last += sg([&](i64 x, i64 y) { return x + XL * b < Np && y + 16 * a < rlast; });
        }
    Out o(v);
    o.op(0, 0, uG * (u64)NT * 8 * uNB, uG * (u64)NW * 8 * uNB);
    o.op(0, 2, uG * (u64)NT * 8 * uNB * uQ * 2, uG * (u64)NW * 8 * uNB * uQ * 2);
    auto site = [&](const char *tag, int mem, int dir, bool vec, i64 l0, i64 l1, i64 g0, i64 g1, i64 loop, u64 wi,
                    u64 sgc, u64 foot) {
        Site x{};
        x.tag = tag; x.mem = mem; x.dir = dir; x.dtype = vec ? "float32x2" : "float32"; x.dsize = vec ? 8 : 4;
        x.nl = 2; x.l[0] = l0; x.l[1] = l1; x.ng = 2; x.g[0] = g0; x.g[1] = g1; x.loop = loop;
        x.wi = wi; x.sg = sgc; x.foot = foot;
        o.site(x);
    };
    if (even)
        site("dgt-D", GL, LD, true, 1, Np / 2, Np * Np / 2, 0, XL, uG * uNp * uQ, uG * sg_D, 3 * uNp * uQ);
    else
        site("dgt-D", GL, LD, false, 2, Np, Np * Np, 0, 1, uG * uNp * uNp, uG * sg_D, 3 * uNp * uNp);
    site("dgt-Dt", LO, ST, true, 1, PD / 2, 0, 0, XL, uG * (u64)NPP * uQ, uG * sg_Dt, (u64)NPP * uQ);
    site("dgt-u", GL, LD, false, 0, 0, 0, 128 * Np, 1, 3 * (u64)Nel * uNp, 3 * (u64)Nel * uNp, (u64)Nel * uNp);
    if (!even) {
        site("dgt-R", LO, LD, false, 2, Np, 0, 0, 1, uG * 128 * uNp, uG * sg_R, 128 * uNp);
        site("dgt-Ur", LO, ST, true, 1, Q, 0, 0, XL, uG * 128 * uQ, uG * sg_Ur, 128 * uQ);
    }
    site("dgt-Us", LO, LD, true, 0, Q, 0, 0, 16 * Q, uG * (u64)NT * 8 * uQ, uG * (u64)NW * 8 * uQ, 128 * uQ);
    site("dgt-Dl", LO, LD, true, PD / 2, 0, 0, 0, XL * PD / 2, uG * (u64)NT * uNB * uQ, uG * (u64)NW * uNB * uQ,
         (u64)NPP * uQ);
    site("dgt-res", GL, ST, false, 1, Np, Nel * Np, 128 * Np, 16 * Np, 3 * (u64)Nel * uNp,
         3 * ((u64)Tfull * sg_res_full + sg_res_last), 3 * (u64)Nel * uNp);
    o.finish(even ? 1 : 2, uG);
    return PM_OK;
}

bool pow2(i64 x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

pm_status validate(const KP &kp) {
    const char *nm = kp.def->name;
    switch (kp.def->fam) {
    case FAM_STREAM: {
        i64 dt = kp.i(0), vec = kp.i(1), N = kp.i(2), s = kp.i(3), L = kp.i(4), shape = kp.i(5), W = kp.i(6);
        if (dt < 0 || dt > 1) return fail(PM_EINVAL, "%s: dtype must be 0 (float32) or 1 (float64)", nm);
        if (vec < 0 || vec > 1) return fail(PM_EINVAL, "%s: vec must be 0 or 1", nm);
        if (L < 1 || L > 4) return fail(PM_EINVAL, "%s: L must be 1..4", nm);
        i64 w = stream_width(dt, vec);
        if (N <= 0 || N % w || N / w > (1LL << 31) - 1)
            return fail(PM_EINVAL, "%s: N must be a positive multiple of %lld below 2^31 vectors", nm, (long long)w);
        i64 M = N / w;
        if (shape == 0) {
            if (!pow2(s) || s > 1024) return fail(PM_EINVAL, "%s: s must be a power of two <= 1024", nm);
            if (M % (256 * s)) return fail(PM_EINVAL, "%s: N/%lld must be a multiple of 256*s", nm, (long long)w);
        } else if (shape == 1) {
            if (W < 16 || W % 16) return fail(PM_EINVAL, "%s: W must be a positive multiple of 16", nm);
            if (M % (16 * W)) return fail(PM_EINVAL, "%s: N/%lld must be a multiple of 16*W", nm, (long long)w);
        } else
            return fail(PM_EINVAL, "%s: shape must be 0 or 1", nm);
        return PM_OK;
    }
    case FAM_FMA:
        if (kp.i(0) < 0 || kp.i(0) > 1) return fail(PM_EINVAL, "%s: dtype must be 0 or 1", nm);
        if (kp.def->variant == 0 && (kp.i(1) < 0 || kp.i(1) > 2)) return fail(PM_EINVAL, "%s: op must be 0 (add), 1 (mul), 2 (madd)", nm);
        if (kp.i(2) < 32 || kp.i(2) % 32 || kp.i(2) > (1LL << 30))
            return fail(PM_EINVAL, "%s: F must be a positive multiple of 32", nm);
        if (kp.i(3) < 1 || kp.i(3) > (1LL << 23)) return fail(PM_EINVAL, "%s: G must be 1..2^23", nm);
        return PM_OK;
    case FAM_SMEM:
        if (kp.i(0) < 4 || kp.i(0) % 4 || kp.i(0) > (1LL << 30))
            return fail(PM_EINVAL, "%s: R must be a positive multiple of 4", nm);
        if (kp.i(1) < 0 || kp.i(1) > 1) return fail(PM_EINVAL, "%s: sync must be 0 or 1", nm);
        if (kp.i(2) < 1 || kp.i(2) > (1LL << 23)) return fail(PM_EINVAL, "%s: G must be 1..2^23", nm);
        return PM_OK;
    case FAM_SMEM2D:
        if (kp.i(0) < 4 || kp.i(0) % 4 || kp.i(0) > (1LL << 30))
            return fail(PM_EINVAL, "%s: R must be a positive multiple of 4", nm);
        if (kp.i(1) != 16 && kp.i(1) != 18) return fail(PM_EINVAL, "%s: T must be 16 or 18", nm);
        if (kp.i(2) < 1 || kp.i(2) > (1LL << 23)) return fail(PM_EINVAL, "%s: G must be 1..2^23", nm);
        return PM_OK;
    case FAM_BARRIER:
        if (kp.i(0) < 0 || kp.i(0) > (1LL << 30)) return fail(PM_EINVAL, "%s: B must be >= 0", nm);
        if (kp.i(1) < 1 || kp.i(1) > (1LL << 23)) return fail(PM_EINVAL, "%s: G must be 1..2^23", nm);
        return PM_OK;
    case FAM_OVERLAP:
        if (kp.i(0) < 0 || kp.i(0) > (1LL << 30)) return fail(PM_EINVAL, "%s: m must be >= 0", nm);
        if (kp.i(1) < 256 || kp.i(1) % 256 || kp.i(1) > (1LL << 31))
            return fail(PM_EINVAL, "%s: N must be a positive multiple of 256", nm);
        return PM_OK;
    case FAM_EMPTY:
        if (kp.i(0) < 1 || kp.i(0) > (1LL << 31) - 1) return fail(PM_EINVAL, "%s: G must be 1..2^31-1", nm);
        return PM_OK;
    case FAM_MM:
        if (kp.i(0) < 16 || kp.i(0) % 16 || kp.i(0) > 32768)
            return fail(PM_EINVAL, "%s: n must be a multiple of 16 in [16, 32768]", nm);
        return PM_OK;
    case FAM_DG: {
        i64 Np = kp.i(0), Nel = kp.i(1), L0 = kp.i(2), L1 = kp.i(3);
        if (!((L0 == 16 && L1 == 16) || (L0 == 32 && L1 == 8)))
            return fail(PM_EINVAL, "%s: work-group (L0, L1) must be (16, 16) or (32, 8)", nm);
        if (Np < 1 || Np > 512) return fail(PM_EINVAL, "%s: Np must be 1..512", nm);
        if (Nel < L0 || Nel % L0 || Nel > (1LL << 24))
            return fail(PM_EINVAL, "%s: Nel must be a positive multiple of L0 (<= 2^24)", nm);
        if ((kp.def->variant == 7 || kp.def->variant == 9) && L0 != L1)
            return fail(PM_EINVAL, "%s: the u-prefetch variant needs a square work-group (16, 16)", nm);
        return PM_OK;
    }
    case FAM_FD:
        if (kp.i(0) < 1 || kp.i(0) > 46000) return fail(PM_EINVAL, "%s: n must be 1..46000", nm);
        return PM_OK;
    case FAM_DGC: {
        const i64 Np = kp.i(0), Nel = kp.i(1), P = kp.i(2);
        if (Np != 4 && Np != 10 && Np != 20 && Np != 35 && Np != 56 && Np != 84)
            return fail(PM_EINVAL, "%s: Np must be 4, 10, 20, 35, 56 or 84", nm);
        if (Nel < 4 || Nel % 4 || Nel > (1LL << 24))
            return fail(PM_EINVAL, "%s: Nel must be a positive multiple of 4 (<= 2^24)", nm);
        if (P < 0 || P > 4096) return fail(PM_EINVAL, "%s: P must be 0 (default) or 1..4096", nm);
        if (kp.i(3) < -1 || kp.i(3) > 1) return fail(PM_EINVAL, "%s: A must be -1 (default), 0 or 1", nm);
        return PM_OK;
    }
    case FAM_DGT:
        if (kp.i(0) < 1 || kp.i(0) > 96) return fail(PM_EINVAL, "%s: Np must be 1..96", nm);
        if (kp.i(1) < 4 || kp.i(1) % 4 || kp.i(1) > 65535LL * 128)
            return fail(PM_EINVAL, "%s: Nel must be a positive multiple of 4 (<= 65535 x 128)", nm);
        return PM_OK;
    case FAM_FDB: {
        i64 n = kp.i(0), BX = kp.i(1), BY = kp.i(2);
        if (BX != 32 && BX != 64 && BX != 128) return fail(PM_EINVAL, "%s: BX must be 32, 64 or 128", nm);
        if (kp.i(5) != 4 && kp.i(5) != 8) return fail(PM_EINVAL, "%s: V must be 4 or 8", nm);
        if (BY != 4 && BY != 8 && BY != 16 && BY != 32) return fail(PM_EINVAL, "%s: BY must be 4, 8, 16 or 32", nm);
        if (n < BX || n % BX || n % BY || n > 46000)
            return fail(PM_EINVAL, "%s: n (<= 46000) must be divisible by BX and BY", nm);
        return PM_OK;
    }
    case FAM_TC:
        if (kp.i(0) < 256 || kp.i(0) % 256 || kp.i(0) > 32768)
            return fail(PM_EINVAL, "%s: n must be a multiple of 256 in [256, 32768]", nm);
        if (kp.def->variant == 0 && (kp.i(1) < 0 || kp.i(1) > 2))
            return fail(PM_EINVAL, "%s: pipe must be 0 (4 stages, 1 CTA/SM), 1 (2 stages, 2 CTAs/SM) or 2 (persistent)",
                        nm);
        return PM_OK;
    case FAM_SIMT: {
        i64 n = kp.i(0), BM = kp.i(1), BN = kp.i(2), BK = kp.i(3);
        bool okm = BM == 64 || BM == 96 || BM == 128 || BM == 256;
        bool okn = BN == 64 || BN == 128 || BN == 256;
        if (!okm || !okn || (BK != 32 && BK != 64))
            return fail(PM_EINVAL, "%s: tile must have BM in {64,96,128,256}, BN in {64,128,256}, BK in {32,64}", nm);
        if (n < 1 || n > 32768 || n % BM || n % BN || n % BK)
            return fail(PM_EINVAL, "%s: n (<= 32768) must be divisible by BM, BN and BK", nm);
        return PM_OK;
    }
    }
    return fail(PM_EINVAL, "unknown family");
}

pm_status counts(const KP &kp, std::vector<pm_feature> &out) {
    pm_status s = validate(kp);
    if (s) return s;
    switch (kp.def->fam) {
    case FAM_STREAM: return counts_stream(kp, out);
    case FAM_FMA: return counts_fma(kp, out);
    case FAM_SMEM: return counts_smem(kp, out);
    case FAM_SMEM2D: return counts_smem2d(kp, out);
    case FAM_BARRIER: return counts_barrier(kp, out);
    case FAM_OVERLAP: return counts_overlap(kp, out);
    case FAM_EMPTY: return counts_empty(kp, out);
    case FAM_MM: return counts_mm(kp, out);
    case FAM_DG: return counts_dg(kp, out);
    case FAM_FD: return counts_fd(kp, out);
    case FAM_SIMT: return counts_simt(kp, out);
    case FAM_TC: return counts_tc(kp, out);
    case FAM_FDB: return counts_fdb(kp, out);
    case FAM_DGT: return counts_dgt(kp, out);
    case FAM_DGC: return counts_dgc(kp, out);
    }
    return fail(PM_EINVAL, "unknown family");
}

pm_status buffers(const KP &kp, std::vector<BufSpec> &b) {
    int var = kp.def->variant;
    switch (kp.def->fam) {
    case FAM_STREAM: {
        int dt = (int)kp.i(0);
        uint64_t N = (uint64_t)kp.i(2);
        static const char *nm[4] = {"in0", "in1", "in2", "in3"};
        for (int a = 0; a < kp.i(4); a++) b.push_back({nm[a], dt, PM_IN, N});
        b.push_back({"out", dt, PM_OUT, N});
        break;
    }
    case FAM_FMA: {
        uint64_t T = (uint64_t)kp.i(3) * 256;
        b.push_back({"seed", (int)kp.i(0), PM_IN, T});
        b.push_back({"out", (int)kp.i(0), PM_OUT, T});
        break;
    }
    case FAM_SMEM2D: {
        uint64_t n = (uint64_t)kp.i(2) * (uint64_t)kp.i(1) * (uint64_t)kp.i(1);
        b.push_back({"in", PM_F32, PM_IN, n});
        b.push_back({"out", PM_F32, PM_OUT, n});
        break;
    }
    case FAM_SMEM: case FAM_BARRIER: {
        uint64_t T = (uint64_t)kp.i(kp.def->fam == FAM_SMEM ? 2 : 1) * 256;
        b.push_back({"in", PM_F32, PM_IN, T});
        b.push_back({"out", PM_F32, PM_OUT, T});
        break;
    }
    case FAM_OVERLAP:
        b.push_back({"in", PM_F32, PM_IN, (uint64_t)kp.i(1)});
        b.push_back({"out", PM_F32, PM_OUT, (uint64_t)kp.i(1)});
        break;
    case FAM_EMPTY: break;
    case FAM_MM: {
        uint64_t N2 = (uint64_t)kp.i(0) * (uint64_t)kp.i(0);
        if (var <= 1) {
            b.push_back({"a", PM_F32, PM_IN, N2});
            b.push_back({"b", PM_F32, PM_IN, N2});
            b.push_back({"c", PM_F32, PM_OUT, N2});
        } else {
            b.push_back({(var == 2 || var == 4) ? "a" : "b", PM_F32, PM_IN, N2});
            b.push_back({"tgt_dest", PM_F32, PM_OUT, N2});
        }
        break;
    }
    case FAM_DG: {
        uint64_t Np = (uint64_t)kp.i(0), Nel = (uint64_t)kp.i(1), L1 = (uint64_t)kp.i(3);
        uint64_t rows = (uint64_t)cdiv((i64)Np, (i64)L1) * L1;
        if (var <= 1 || var == 7 || var == 8) {   // dmPF-T: u as uT[j, k], res as resT[m, i, k]
            b.push_back({"diff_mat", PM_F32, PM_IN, 3 * Np * Np});
            b.push_back({"u", PM_F32, PM_IN, Nel * Np});
            b.push_back({"res", PM_F32, PM_OUT, 3 * Nel * Np});
        } else if (var == 2 || var == 4 || var == 9 || var == 10) {
            b.push_back({"u", PM_F32, PM_IN, Nel * Np});
            b.push_back({"tgt_dest", PM_F32, PM_OUT, rows * Nel});
        } else if (var == 3 || var == 5) {
            b.push_back({"diff_mat", PM_F32, PM_IN, 3 * Np * Np});
            b.push_back({"tgt_dest", PM_F32, PM_OUT, rows * Nel});
        } else {
            b.push_back({"res", PM_F32, PM_OUT, 3 * Nel * Np});
        }
        break;
    }
    case FAM_DGT:
    case FAM_DGC: {
        uint64_t Np = (uint64_t)kp.i(0), Nel = (uint64_t)kp.i(1);
        b.push_back({"diff_mat", PM_F32, PM_IN, 3 * Np * Np});
        b.push_back({"u", PM_F32, PM_IN, Nel * Np});
        b.push_back({"res", PM_F32, PM_OUT, 3 * Nel * Np});
        break;
    }
    case FAM_FDB: {
        uint64_t n = (uint64_t)kp.i(0);
        b.push_back({"u", PM_F32, PM_IN, (n + 2) * (n + 4)});
        b.push_back({"res", PM_F32, PM_OUT, n * n});
        break;
    }
    case FAM_TC: {
        uint64_t N2 = (uint64_t)kp.i(0) * (uint64_t)kp.i(0);
        b.push_back({"a", PM_BF16, PM_IN, N2});
        b.push_back({"bt", PM_BF16, PM_IN, N2});
        b.push_back({"c", PM_F32, PM_OUT, N2});
        break;
    }
    case FAM_SIMT: {
        uint64_t N2 = (uint64_t)kp.i(0) * (uint64_t)kp.i(0);
        b.push_back({"a", PM_F32, PM_IN, N2});
        b.push_back({"b", PM_F32, PM_IN, N2});
        b.push_back({"c", PM_F32, PM_OUT, N2});
        break;
    }
    case FAM_FD: {
        uint64_t n = (uint64_t)kp.i(0), W = n + 2;
        uint64_t Gt = (uint64_t)cdiv((i64)n, 14), Gd = (uint64_t)cdiv((i64)n, 16);
        if (var == 0 || var == 1 || var == 6) {
            b.push_back({"u", PM_F32, PM_IN, W * W});
            b.push_back({"res", PM_F32, PM_OUT, n * n});
        } else if (var == 2 || var == 4 || var == 7) {
            uint64_t G = var == 2 ? Gt : Gd, T = var == 7 ? 18 : 16;
            b.push_back({"u", PM_F32, PM_IN, W * W});
            b.push_back({"tgt_dest", PM_F32, PM_OUT, T * T * G * G});
        } else {
            b.push_back({"res", PM_F32, PM_OUT, n * n});
        }
        break;
    }
    }
    return PM_OK;
}

}  // namespace pm
