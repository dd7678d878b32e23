// Feature counts of a kernel given as an affine loop-nest description
// (pm_counts_desc): the counting the paper delegates to a polyhedral library
// (Section "Gathering Kernel Statistics", Algorithm 1, Algorithm 2), for
// kernels that are not in the registry.
//
// A description names the size parameters, the grid and work-group extents,
// and a list of statements.  Each statement has its own loop nest (bounds are
// integer expressions of the parameters, the thread indices g0..g2, l0..l2
// and the enclosing loop variables; the upper bound is exclusive), guards
// (expressions that must be >= 0), scalar operation counts, and access sites
// with affine index expressions; a "barrier" statement is a local barrier.
//
// At given parameter values the statements are executed for every work-item
// and every loop point: arithmetic and local accesses count per sub-group
// instance (32 consecutive linear thread ids; an instance counts once if any
// lane executes it), global accesses per work-item unless their lid(0)
// stride is 0, barriers per work-item (equal for all), footprints as the
// number of distinct indices of a site.  Strides are finite differences,
// checked constant over the domain.
//
// Large sizes: counts are quasi-polynomials in each size parameter.  For the
// parameters listed in `interp` (name, period, degree bound) the engine
// enumerates degree + 2 sizes in the target's residue class and extrapolates
// every field exactly with Newton forward differences in 128-bit integers;
// the extra sample must make the (degree + 1)-th difference vanish.
#include <algorithm>
#include <cctype>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <unordered_set>
#include <vector>

#include "pm_internal.h"

namespace pm {
namespace {

typedef int64_t i64;
typedef uint64_t u64;

// ---------------------------------------------------------------- expressions
// Compiled to a small stack program over variable slots.
enum Op { PUSH, VAR, ADD, SUB, MUL, DIV, MOD, NEG, MIN, MAX };
struct Ins {
    Op op;
    i64 v;
};
struct Expr {
    std::vector<Ins> code;
    i64 eval(const i64 *vars) const {
        i64 st[64];
        int sp = 0;
        for (const Ins &c : code) {
            switch (c.op) {
            case PUSH: st[sp++] = c.v; break;
            case VAR: st[sp++] = vars[c.v]; break;
            case NEG: st[sp - 1] = -st[sp - 1]; break;
            default: {
                i64 b = st[--sp], a = st[sp - 1], r = 0;
                switch (c.op) {
                case ADD: r = a + b; break;
                case SUB: r = a - b; break;
                case MUL: r = a * b; break;
                case DIV: r = b ? (a / b - ((a % b != 0) && ((a < 0) != (b < 0)))) : 0; break;   // floor
                case MOD: r = b ? a - b * (a / b - ((a % b != 0) && ((a < 0) != (b < 0)))) : 0; break;
                case MIN: r = a < b ? a : b; break;
                case MAX: r = a > b ? a : b; break;
                default: break;
                }
                st[sp - 1] = r;
            }
            }
        }
        return sp ? st[0] : 0;
    }
};

struct Parser {
    const std::string &s;
    size_t i = 0;
    const std::map<std::string, int> &slots;
    std::string err;
    Expr e;
    int depth = 0, maxdepth = 0;
    Parser(const std::string &src, const std::map<std::string, int> &sl) : s(src), slots(sl) {}
    void ws() {
        while (i < s.size() && isspace((unsigned char)s[i])) i++;
    }
    void emit(Op o, i64 v = 0) {
        e.code.push_back({o, v});
        depth += (o == PUSH || o == VAR) ? 1 : (o == NEG ? 0 : -1);
        if (depth > maxdepth) maxdepth = depth;
    }
    bool primary() {
        ws();
        if (i >= s.size()) return fail_at("unexpected end");
        if (s[i] == '(') {
            i++;
            if (!sum()) return false;
            ws();
            if (i >= s.size() || s[i] != ')') return fail_at("missing ')'");
            i++;
            return true;
        }
        if (s[i] == '-') {
            i++;
            if (!primary()) return false;
            emit(NEG);
            return true;
        }
        if (isdigit((unsigned char)s[i])) {
            i64 v = 0;
            while (i < s.size() && isdigit((unsigned char)s[i])) v = v * 10 + (s[i++] - '0');
            emit(PUSH, v);
            return true;
        }
        if (isalpha((unsigned char)s[i]) || s[i] == '_') {
            size_t j = i;
            while (i < s.size() && (isalnum((unsigned char)s[i]) || s[i] == '_')) i++;
            std::string name = s.substr(j, i - j);
            if (name == "min" || name == "max") {
                ws();
                if (i >= s.size() || s[i] != '(') return fail_at("min/max need '('");
                i++;
                if (!sum()) return false;
                ws();
                if (i >= s.size() || s[i] != ',') return fail_at("min/max need two arguments");
                i++;
                if (!sum()) return false;
                ws();
                if (i >= s.size() || s[i] != ')') return fail_at("missing ')'");
                i++;
                emit(name == "min" ? MIN : MAX);
                return true;
            }
            auto it = slots.find(name);
            if (it == slots.end()) return fail_at(("unknown name '" + name + "'").c_str());
            emit(VAR, it->second);
            return true;
        }
        return fail_at("unexpected character");
    }
    bool product() {
        if (!primary()) return false;
        for (;;) {
            ws();
            if (i < s.size() && (s[i] == '*' || s[i] == '/' || s[i] == '%')) {
                char c = s[i++];
                if (!primary()) return false;
                emit(c == '*' ? MUL : c == '/' ? DIV : MOD);
            } else {
                return true;
            }
        }
    }
    bool sum() {
        if (!product()) return false;
        for (;;) {
            ws();
            if (i < s.size() && (s[i] == '+' || s[i] == '-')) {
                char c = s[i++];
                if (!product()) return false;
                emit(c == '+' ? ADD : SUB);
            } else {
                return true;
            }
        }
    }
    bool fail_at(const char *m) {
        if (err.empty()) err = std::string(m) + " at offset " + std::to_string(i) + " in '" + s + "'";
        return false;
    }
    bool run() {
        if (!sum()) return false;
        ws();
        if (i != s.size()) return fail_at("trailing text");
        if (maxdepth > 60) return fail_at("expression too deep");
        return true;
    }
};

// ---------------------------------------------------------------- description
constexpr int MAXL = 6;   // loops per statement
struct Access {
    std::string tag, dtype;
    int mem, dir, dsize;
    Expr idx;
};
struct Stmt {
    bool barrier = false;
    int nloop = 0;
    std::string lname[MAXL];
    Expr lo[MAXL], hi[MAXL];
    std::vector<Expr> guards;
    std::string dt = "float32";
    int nop[3] = {0, 0, 0};
    std::vector<Access> acc;
};
struct Desc {
    std::vector<std::string> params;
    int ng = 0, nl = 0;
    Expr grid[3], group[3];
    std::vector<Stmt> st;
};
// variable slots: params, then g0 g1 g2 l0 l1 l2, then the statement's loops
constexpr int NTH = 6;

std::vector<std::string> words(const std::string &line, size_t n, std::string *rest) {
    std::vector<std::string> w;
    size_t i = 0;
    while (w.size() < n) {
        while (i < line.size() && isspace((unsigned char)line[i])) i++;
        if (i >= line.size()) break;
        size_t j = i;
        while (j < line.size() && !isspace((unsigned char)line[j])) j++;
        w.push_back(line.substr(i, j - i));
        i = j;
    }
    if (rest) {
        while (i < line.size() && isspace((unsigned char)line[i])) i++;
        *rest = line.substr(i);
    }
    return w;
}

pm_status compile(const std::string &src, const std::map<std::string, int> &slots, Expr *out, int lineno) {
    Parser p(src, slots);
    if (!p.run()) return fail(PM_EPARSE, "kernel description line %d: %s", lineno, p.err.c_str());
    *out = p.e;
    return PM_OK;
}

pm_status parse_desc(const char *text, Desc &d) {
    std::map<std::string, int> base;
    static const char *th[NTH] = {"g0", "g1", "g2", "l0", "l1", "l2"};
    std::vector<std::string> lines;
    {
        std::string cur;
        for (const char *c = text; *c; c++) {
            if (*c == '\n') { lines.push_back(cur); cur.clear(); }
            else cur += *c;
        }
        lines.push_back(cur);
    }
    Stmt *cur = nullptr;
    std::map<std::string, int> slots;
    std::unordered_set<std::string> tags;
    pm_status s;
    for (size_t ln = 0; ln < lines.size(); ln++) {
        std::string line = lines[ln];
        size_t h = line.find('#');
        if (h != std::string::npos) line = line.substr(0, h);
        std::string rest;
        std::vector<std::string> w = words(line, 1, &rest);
        if (w.empty()) continue;
        const std::string &k = w[0];
        const int lno = (int)ln + 1;
        if (k == "params") {
            if (!d.params.empty() || !d.st.empty()) return fail(PM_EPARSE, "kernel description line %d: params must come first, once", lno);
            std::vector<std::string> p = words(rest, 64, nullptr);
            for (auto &n : p) {
                if (base.count(n)) return fail(PM_EPARSE, "kernel description line %d: duplicate name '%s'", lno, n.c_str());
                base[n] = (int)d.params.size();
                d.params.push_back(n);
            }
            for (int t = 0; t < NTH; t++) base[th[t]] = (int)d.params.size() + t;
        } else if (k == "grid" || k == "group") {
            if (d.params.empty() && base.empty())
                for (int t = 0; t < NTH; t++) base[th[t]] = t;
            std::vector<std::string> e = words(rest, 4, nullptr);
            if (e.empty() || e.size() > 3) return fail(PM_EPARSE, "kernel description line %d: %s needs 1 to 3 extents", lno, k.c_str());
            std::map<std::string, int> pslots;
            for (size_t a = 0; a < d.params.size(); a++) pslots[d.params[a]] = (int)a;
            Expr *dst = k == "grid" ? d.grid : d.group;
            for (size_t a = 0; a < e.size(); a++)
                if ((s = compile(e[a], pslots, &dst[a], lno))) return s;
            for (size_t a = e.size(); a < 3; a++) dst[a].code = {{PUSH, 1}};
            (k == "grid" ? d.ng : d.nl) = (int)e.size();
        } else if (k == "stmt" || k == "barrier") {
            if (!d.ng || !d.nl) return fail(PM_EPARSE, "kernel description line %d: grid and group come before statements", lno);
            d.st.emplace_back();
            cur = &d.st.back();
            cur->barrier = k == "barrier";
            slots = base;
        } else {
            if (!cur) return fail(PM_EPARSE, "kernel description line %d: '%s' outside a statement", lno, k.c_str());
            if (k == "loop") {
                std::vector<std::string> e = words(rest, 3, nullptr);
                if (e.size() != 3) return fail(PM_EPARSE, "kernel description line %d: loop <var> <lo> <hi>", lno);
                if (cur->nloop >= MAXL) return fail(PM_EPARSE, "kernel description line %d: more than %d loops", lno, MAXL);
                if (slots.count(e[0])) return fail(PM_EPARSE, "kernel description line %d: name '%s' in use", lno, e[0].c_str());
                const int li = cur->nloop;
                if ((s = compile(e[1], slots, &cur->lo[li], lno)) || (s = compile(e[2], slots, &cur->hi[li], lno))) return s;
                cur->lname[li] = e[0];
                slots[e[0]] = (int)d.params.size() + NTH + li;
                cur->nloop++;
            } else if (k == "guard") {
                cur->guards.emplace_back();
                if ((s = compile(rest, slots, &cur->guards.back(), lno))) return s;
            } else if (k == "ops") {
                std::vector<std::string> e = words(rest, 4, nullptr);
                if (e.size() != 4 || cur->barrier) return fail(PM_EPARSE, "kernel description line %d: ops <dtype> <add> <mul> <madd>", lno);
                if (e[0] != "float32" && e[0] != "float64" && e[0] != "bfloat16")
                    return fail(PM_EPARSE, "kernel description line %d: op dtype must be float32, float64 or bfloat16", lno);
                cur->dt = e[0];
                for (int o = 0; o < 3; o++) cur->nop[o] = atoi(e[1 + o].c_str());
            } else if (k == "access") {
                std::vector<std::string> e = words(rest, 5, &rest);
                if (e.size() != 5 || rest.empty() || cur->barrier)
                    return fail(PM_EPARSE, "kernel description line %d: access <tag> <global|local> <load|store> <dtype> <bytes> <index>", lno);
                Access a;
                a.tag = e[0];
                if (a.tag.size() >= 32) return fail(PM_EPARSE, "kernel description line %d: tag too long", lno);
                if (!tags.insert(a.tag).second) return fail(PM_EPARSE, "kernel description line %d: duplicate tag '%s'", lno, a.tag.c_str());
                if (e[1] != "global" && e[1] != "local") return fail(PM_EPARSE, "kernel description line %d: global or local", lno);
                if (e[2] != "load" && e[2] != "store") return fail(PM_EPARSE, "kernel description line %d: load or store", lno);
                a.mem = e[1] == "local";
                a.dir = e[2] == "store";
                a.dtype = e[3];
                a.dsize = atoi(e[4].c_str());
                if (a.dtype.size() >= 16 || a.dsize <= 0) return fail(PM_EPARSE, "kernel description line %d: bad data type or size", lno);
                if ((s = compile(rest, slots, &a.idx, lno))) return s;
                cur->acc.push_back(a);
            } else {
                return fail(PM_EPARSE, "kernel description line %d: unknown keyword '%s'", lno, k.c_str());
            }
        }
    }
    if (!d.ng || !d.nl) return fail(PM_EPARSE, "kernel description: grid and group are required");
    return PM_OK;
}

// ---------------------------------------------------------------- enumeration
struct VecHash {
    size_t operator()(const std::vector<i64> &v) const {
        uint64_t h = 1469598103934665603ull;
        for (i64 x : v) h = (h ^ (uint64_t)x) * 1099511628211ull + 0x9E3779B97F4A7C15ull;
        return (size_t)(h ^ (h >> 29));
    }
};
struct SiteStat {
    u64 wi = 0, sg = 0;
    std::unordered_set<i64> foot;
    bool have = false, affine = true;
    i64 ls[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, loop = 0;
};

struct Enum {
    const Desc &d;
    std::vector<i64> vars;
    u64 op_wi[3][3] = {{0}}, op_sg[3][3] = {{0}};
    std::vector<std::vector<SiteStat>> ss;   // per statement, per access
    std::unordered_set<std::vector<i64>, VecHash> sgset;
    i64 bar_cur = 0, bar_min = -1, bar_max = -1;
    u64 budget;
    std::string err;
    explicit Enum(const Desc &dd, u64 b) : d(dd), budget(b) {
        ss.resize(d.st.size());
        for (size_t k = 0; k < d.st.size(); k++) ss[k].resize(d.st[k].acc.size());
    }
    static int dti(const std::string &t) { return t == "float32" ? 0 : t == "float64" ? 1 : 2; }

    void instance(size_t k, int np) {
        const Stmt &S = d.st[k];
        if (budget == 0) { err = "enumeration budget exhausted (use interpolation for this size)"; return; }
        budget--;
        if (S.barrier) { bar_cur++; return; }
        std::vector<i64> key(1 + S.nloop);
        key[0] = (i64)k;
        for (int i = 0; i < S.nloop; i++) key[1 + i] = vars[np + NTH + i];
        const bool fresh = sgset.insert(key).second;
        const int dt = dti(S.dt);
        for (int o = 0; o < 3; o++) {
            op_wi[dt][o] += (u64)S.nop[o];
            if (fresh) op_sg[dt][o] += (u64)S.nop[o];
        }
        for (size_t a = 0; a < S.acc.size(); a++) {
            const Expr &e = S.acc[a].idx;
            SiteStat &t = ss[k][a];
            const i64 base = e.eval(vars.data());
            t.wi++;
            if (fresh) t.sg++;
            t.foot.insert(base);
            i64 ls[3], gs[3], lp = 0;
            for (int ax = 0; ax < 3; ax++) {
                vars[np + 3 + ax]++;
                ls[ax] = e.eval(vars.data()) - base;
                vars[np + 3 + ax]--;
                vars[np + ax]++;
                gs[ax] = e.eval(vars.data()) - base;
                vars[np + ax]--;
            }
            if (S.nloop) {
                vars[np + NTH + S.nloop - 1]++;
                lp = e.eval(vars.data()) - base;
                vars[np + NTH + S.nloop - 1]--;
            }
            if (!t.have) {
                for (int ax = 0; ax < 3; ax++) { t.ls[ax] = ls[ax]; t.gs[ax] = gs[ax]; }
                t.loop = lp;
                t.have = true;
            } else {
                for (int ax = 0; ax < 3; ax++)
                    if (t.ls[ax] != ls[ax] || t.gs[ax] != gs[ax]) t.affine = false;
                if (t.loop != lp) t.affine = false;
            }
        }
    }
    void loops(size_t k, int li, int np) {
        const Stmt &S = d.st[k];
        if (!err.empty()) return;
        if (li == S.nloop) {
            for (const Expr &g : S.guards)
                if (g.eval(vars.data()) < 0) return;
            instance(k, np);
            return;
        }
        const i64 lo = S.lo[li].eval(vars.data()), hi = S.hi[li].eval(vars.data());
        for (i64 v = lo; v < hi && err.empty(); v++) {
            vars[np + NTH + li] = v;
            loops(k, li + 1, np);
        }
    }
    pm_status run(const std::vector<i64> &pv, i64 G[3], i64 L[3]) {
        const int np = (int)pv.size();
        vars.assign(np + NTH + MAXL, 0);
        for (int i = 0; i < np; i++) vars[i] = pv[i];
        const i64 T = L[0] * L[1] * L[2];
        for (i64 g2 = 0; g2 < G[2]; g2++)
            for (i64 g1 = 0; g1 < G[1]; g1++)
                for (i64 g0 = 0; g0 < G[0]; g0++)
                    for (i64 q = 0; q * 32 < T; q++) {
                        sgset.clear();
                        for (i64 t = q * 32; t < q * 32 + 32 && t < T; t++) {
                            vars[np] = g0; vars[np + 1] = g1; vars[np + 2] = g2;
                            vars[np + 3] = t % L[0]; vars[np + 4] = (t / L[0]) % L[1]; vars[np + 5] = t / (L[0] * L[1]);
                            bar_cur = 0;
                            for (size_t k = 0; k < d.st.size(); k++) loops(k, 0, np);
                            if (!err.empty()) return fail(PM_EINVAL, "pm_counts_desc: %s", err.c_str());
                            if (bar_min < 0 || bar_cur < bar_min) bar_min = bar_cur;
                            if (bar_cur > bar_max) bar_max = bar_cur;
                        }
                    }
        if (bar_min != bar_max) return fail(PM_EINVAL, "pm_counts_desc: work-items meet different barrier counts");
        return PM_OK;
    }
};

// one full enumeration at parameter values pv -> feature records (canonical order)
pm_status count_at(const Desc &d, const std::vector<i64> &pv, u64 budget, std::vector<pm_feature> &out) {
    i64 G[3], L[3];
    for (int a = 0; a < 3; a++) {
        G[a] = d.grid[a].eval(pv.data());
        L[a] = d.group[a].eval(pv.data());
        if (G[a] < 1 || L[a] < 1) return fail(PM_EINVAL, "pm_counts_desc: grid and group extents must be >= 1");
    }
    if (L[0] * L[1] * L[2] > 1024) return fail(PM_EINVAL, "pm_counts_desc: more than 1024 work-items per group");
    Enum en(d, budget);
    pm_status s = en.run(pv, G, L);
    if (s) return s;
    out.clear();
    static const char *dtn[3] = {"float32", "float64", "bfloat16"};
    static const char *opn[3] = {"add", "mul", "madd"};
    for (int dt = 0; dt < 3; dt++)
        for (int o = 0; o < 3; o++)
            if (en.op_wi[dt][o]) {
                pm_feature f;
                memset(&f, 0, sizeof f);
                f.kind = PM_FEAT_OP;
                f.gran = PM_GRAN_SG;
                f.count = f.count_sg = en.op_sg[dt][o];
                f.count_wi = en.op_wi[dt][o];
                snprintf(f.dtype, sizeof f.dtype, "%s", dtn[dt]);
                snprintf(f.op, sizeof f.op, "%s", opn[o]);
                out.push_back(f);
            }
    for (size_t k = 0; k < d.st.size(); k++)
        for (size_t a = 0; a < d.st[k].acc.size(); a++) {
            const Access &A = d.st[k].acc[a];
            const SiteStat &t = en.ss[k][a];
            if (!t.wi) continue;
            if (!t.affine) return fail(PM_EINVAL, "pm_counts_desc: access '%s' is not affine", A.tag.c_str());
            pm_feature f;
            memset(&f, 0, sizeof f);
            f.kind = PM_FEAT_MEM;
            snprintf(f.tag, sizeof f.tag, "%s", A.tag.c_str());
            snprintf(f.dtype, sizeof f.dtype, "%s", A.dtype.c_str());
            f.mem = A.mem;
            f.dir = A.dir;
            f.dsize = A.dsize;
            f.nl = d.nl;
            f.ng = d.ng;
            for (int ax = 0; ax < 3; ax++) {
                f.lstride[ax] = ax < d.nl ? t.ls[ax] : 0;
                f.gstride[ax] = ax < d.ng ? t.gs[ax] : 0;
            }
            f.loop_stride = t.loop;
            f.count_wi = f.accesses = t.wi;
            f.count_sg = t.sg;
            f.footprint = t.foot.size();
            const bool per_sg = A.mem == 1 || f.lstride[0] == 0;
            f.gran = per_sg ? PM_GRAN_SG : PM_GRAN_WI;
            f.count = per_sg ? t.sg : t.wi;
            out.push_back(f);
        }
    pm_feature f;
    memset(&f, 0, sizeof f);
    f.kind = PM_FEAT_SYNC;
    f.gran = PM_GRAN_WI;
    f.count = (u64)(en.bar_max < 0 ? 0 : en.bar_max);
    out.push_back(f);
    f.kind = PM_FEAT_GROUPS;
    f.gran = PM_GRAN_WG;
    f.count = (u64)(G[0] * G[1] * G[2]);
    out.push_back(f);
    f.kind = PM_FEAT_LAUNCH;
    f.gran = PM_GRAN_K;
    f.count = 1;
    out.push_back(f);
    return PM_OK;
}

// ---------------------------------------------------------------- extrapolation
typedef __int128 i128;
// the numeric fields of a record, as signed 128-bit values
constexpr int NF = 13;
void fields(const pm_feature &f, i128 *x) {
    x[0] = f.count; x[1] = f.count_wi; x[2] = f.count_sg; x[3] = f.accesses; x[4] = f.footprint;
    for (int a = 0; a < 3; a++) { x[5 + a] = f.lstride[a]; x[8 + a] = f.gstride[a]; }
    x[11] = f.loop_stride;
    x[12] = 0;
}
bool set_fields(pm_feature &f, const i128 *x) {
    for (int k = 0; k < 5; k++)
        if (x[k] < 0 || x[k] > (i128)UINT64_MAX) return false;
    for (int k = 5; k < 12; k++)
        if (x[k] < (i128)INT64_MIN || x[k] > (i128)INT64_MAX) return false;
    f.count = (u64)x[0]; f.count_wi = (u64)x[1]; f.count_sg = (u64)x[2]; f.accesses = (u64)x[3];
    f.footprint = (u64)x[4];
    for (int a = 0; a < 3; a++) { f.lstride[a] = (i64)x[5 + a]; f.gstride[a] = (i64)x[8 + a]; }
    f.loop_stride = (i64)x[11];
    return true;
}
bool same_shape(const pm_feature &a, const pm_feature &b) {
    return a.kind == b.kind && a.mem == b.mem && a.dir == b.dir && !strcmp(a.tag, b.tag) && !strcmp(a.dtype, b.dtype) &&
           !strcmp(a.op, b.op) && a.nl == b.nl && a.ng == b.ng && a.gran == b.gran;
}

struct Interp {
    int param;   // index into the description's parameters
    i64 period;
    int degree;
};

// ---------------------------------------------------------------- period and degree
// A bound on how an expression grows with one size parameter P (the other
// parameters fixed at their values): its polynomial degree in P, whether it
// is a known constant (and its value), and the constant divisors and moduli
// applied to P-dependent operands.  A thread index has the degree of its
// extent, a loop variable the larger degree of its bounds.
struct Deg {
    int d;
    bool is_const;
    i64 v;
};

i64 gcd64(i64 a, i64 b) {
    while (b) { const i64 t = a % b; a = b; b = t; }
    return a < 0 ? -a : a;
}

struct Deriver {
    int P, np;
    const std::vector<i64> &pv;
    i64 period = 1;
    std::string err;
    std::vector<int> slot_deg;   // degree of each variable slot (index and loop variables)
    Deriver(int p, const std::vector<i64> &vals) : P(p), np((int)vals.size()), pv(vals) {
        slot_deg.assign(np + NTH + MAXL, 0);
    }
    void divides(i64 c) {
        c = c < 0 ? -c : c;
        if (c <= 1) return;
        period = period / gcd64(period, c) * c;
        if (period > ((i64)1 << 24)) err = "the period in this parameter exceeds 2^24";
    }
    Deg eval(const Expr &e) {
        Deg st[64];
        int sp = 0;
        for (const Ins &c : e.code) {
            if (c.op == PUSH) { st[sp++] = {0, true, c.v}; continue; }
            if (c.op == VAR) {
                const int k = (int)c.v;
                if (k < np) st[sp++] = k == P ? Deg{1, false, 0} : Deg{0, true, pv[k]};
                else st[sp++] = {slot_deg[k], false, 0};
                continue;
            }
            if (c.op == NEG) {
                Deg &a = st[sp - 1];
                if (a.is_const) a.v = -a.v;
                continue;
            }
            const Deg b = st[--sp], a = st[sp - 1];
            Deg r{0, false, 0};
            if (a.is_const && b.is_const) {
                Expr tmp;
                tmp.code = {{PUSH, a.v}, {PUSH, b.v}, c};
                r = {0, true, tmp.eval(nullptr)};
            } else {
                switch (c.op) {
                case ADD: case SUB: case MIN: case MAX: r.d = std::max(a.d, b.d); break;
                case MUL: r.d = a.d + b.d; break;
                case DIV:
                case MOD:
                    if (!b.is_const) {
                        if (a.d > 0 || b.d > 0) err = "a divisor or modulus that is not constant depends on the parameter";
                        r.d = std::max(a.d, b.d);
                    } else {
                        if (a.d > 0) divides(b.v);
                        r.d = c.op == DIV ? a.d : 0;
                    }
                    break;
                default: break;
                }
            }
            st[sp - 1] = r;
        }
        return sp ? st[0] : Deg{0, true, 0};
    }
};

// Period and degree bound of every count of `d` as a quasi-polynomial in
// parameter P (the others at pv): the period is the lcm of the constant
// divisors and moduli applied to P-dependent expressions; the degree bound
// is, over the statements, the larger of the instance-count degree (the
// degrees of the grid extents plus, per loop, the larger degree of its
// bounds: the number of points of the domain, which bounds the footprints,
// sub-group counts and barriers too) and the degrees of the access index
// expressions (their strides).  PM_EINVAL where no such bound follows from
// the description: a work-group extent depending on P (its sub-group
// decomposition then changes with P), or a P-dependent non-constant divisor.
pm_status derive_interp(const Desc &d, int P, const std::vector<i64> &pv, i64 *period, int *degree) {
    Deriver D(P, pv);
    int grid_deg = 0;
    for (int a = 0; a < 3; a++) {
        const Deg g = D.eval(d.grid[a]), l = D.eval(d.group[a]);
        if (l.d > 0 || !l.is_const) return fail(PM_EINVAL, "pm_counts_desc: the work-group extent depends on %s; "
                                                 "state its period and degree", d.params[P].c_str());
        D.slot_deg[D.np + a] = g.d;        // g_a ranges over the grid extent
        D.slot_deg[D.np + 3 + a] = 0;      // l_a over a constant extent
        grid_deg += g.d;
    }
    int deg = grid_deg;
    for (const Stmt &S : d.st) {
        int inst = grid_deg;
        for (int li = 0; li < S.nloop; li++) {
            const int ld = std::max(D.eval(S.lo[li]).d, D.eval(S.hi[li]).d);
            D.slot_deg[D.np + NTH + li] = ld;
            inst += ld;
        }
        for (const Expr &g : S.guards) D.eval(g);
        deg = std::max(deg, inst);
        for (const Access &A : S.acc) deg = std::max(deg, D.eval(A.idx).d);
        for (int li = 0; li < MAXL; li++) D.slot_deg[D.np + NTH + li] = 0;
    }
    if (!D.err.empty()) return fail(PM_EINVAL, "pm_counts_desc: %s (%s); state its period and degree", D.err.c_str(),
                                    d.params[P].c_str());
    if (deg > 10) return fail(PM_EINVAL, "pm_counts_desc: degree bound %d in %s exceeds 10", deg, d.params[P].c_str());
    *period = D.period;
    *degree = deg;
    return PM_OK;
}

pm_status counts_rec(const Desc &d, std::vector<i64> pv, const std::vector<Interp> &ip, size_t level, u64 budget,
                     std::vector<pm_feature> &out) {
    if (level == ip.size()) return count_at(d, pv, budget, out);
    const Interp &I = ip[level];
    const i64 target = pv[I.param];
    i64 rho = ((target % I.period) + I.period) % I.period;
    const i64 x0 = rho + I.period;   // first sample: one period above the residue
    if (target <= x0 + I.period * (I.degree + 2)) return counts_rec(d, pv, ip, level + 1, budget, out);
    const int ns = I.degree + 3;   // degree + 1 samples fix the polynomial, two more check it
    std::vector<std::vector<pm_feature>> smp(ns);
    pm_status s;
    for (int j = 0; j < ns; j++) {
        pv[I.param] = x0 + I.period * j;
        if ((s = counts_rec(d, pv, ip, level + 1, budget, smp[j]))) return s;
        if (smp[j].size() != smp[0].size())
            return fail(PM_EINVAL, "pm_counts_desc: the set of features changes with %s (not one quasi-polynomial)",
                        d.params[I.param].c_str());
        for (size_t r = 0; r < smp[j].size(); r++)
            if (!same_shape(smp[j][r], smp[0][r]))
                return fail(PM_EINVAL, "pm_counts_desc: the features change with %s", d.params[I.param].c_str());
    }
    const i128 t = (target - x0) / I.period;   // target = x0 + period * t
    out = smp[0];
    for (size_t r = 0; r < out.size(); r++) {
        i128 diff[13][NF];   // forward differences, diff[k] = Delta^k at x0
        for (int j = 0; j < ns; j++) fields(smp[j][r], diff[j]);
        for (int k = 1; k < ns; k++)
            for (int j = ns - 1; j >= k; j--)
                for (int f = 0; f < NF; f++) diff[j][f] -= diff[j - 1][f];
        for (int f = 0; f < NF; f++)
            if (diff[ns - 1][f] != 0 || diff[ns - 2][f] != 0)
                return fail(PM_EINVAL, "pm_counts_desc: a count is not a polynomial of degree <= %d in %s on the residue class "
                            "(raise the degree or the period)", I.degree, d.params[I.param].c_str());
        i128 val[NF] = {0}, binom = 1;   // C(t, k)
        for (int k = 0; k <= I.degree; k++) {
            if (k > 0) binom = binom * (t - (k - 1)) / k;
            for (int f = 0; f < NF; f++) val[f] += binom * diff[k][f];
        }
        if (!set_fields(out[r], val)) return fail(PM_EINVAL, "pm_counts_desc: an extrapolated count is out of range");
    }
    return PM_OK;
}

}  // namespace
}  // namespace pm

using namespace pm;

extern "C" pm_status pm_counts_desc(const char *description, const pm_param *p, size_t np, const pm_interp *interp,
                                    size_t ninterp, pm_feature *out, size_t cap, size_t *n_out) {
    if (!description || !n_out) return fail(PM_EINVAL, "pm_counts_desc: NULL argument");
    if ((np && !p) || (ninterp && !interp) || (cap && !out)) return fail(PM_EINVAL, "pm_counts_desc: NULL array");
    Desc d;
    pm_status s = parse_desc(description, d);
    if (s) return s;
    std::vector<i64> pv(d.params.size(), 0);
    std::vector<bool> seen(d.params.size(), false);
    for (size_t i = 0; i < np; i++) {
        size_t k = 0;
        while (k < d.params.size() && (!p[i].key || d.params[k] != p[i].key)) k++;
        if (k == d.params.size()) return fail(PM_EINVAL, "pm_counts_desc: unknown parameter '%s'", p[i].key ? p[i].key : "");
        if (p[i].value != (double)(i64)p[i].value) return fail(PM_EINVAL, "pm_counts_desc: '%s' must be an integer", p[i].key);
        pv[k] = (i64)p[i].value;
        seen[k] = true;
    }
    for (size_t k = 0; k < d.params.size(); k++)
        if (!seen[k]) return fail(PM_EINVAL, "pm_counts_desc: missing parameter '%s'", d.params[k].c_str());
    std::vector<Interp> ip;
    for (size_t i = 0; i < ninterp; i++) {
        size_t k = 0;
        while (k < d.params.size() && (!interp[i].name || d.params[k] != interp[i].name)) k++;
        if (k == d.params.size()) return fail(PM_EINVAL, "pm_counts_desc: interpolation over unknown parameter");
        i64 period = interp[i].period;
        int degree = interp[i].degree;
        if (period == 0 || degree == -1) {   // derive what the caller left open
            i64 dp;
            int dd;
            if ((s = derive_interp(d, (int)k, pv, &dp, &dd))) return s;
            if (period == 0) period = dp;
            if (degree == -1) degree = dd;
        }
        if (period < 1 || degree < 0 || degree > 10)
            return fail(PM_EINVAL, "pm_counts_desc: need period >= 1 and degree 0..10");
        ip.push_back({(int)k, period, degree});
    }
    std::vector<pm_feature> v;
    if ((s = counts_rec(d, pv, ip, 0, (u64)1 << 31, v))) return s;
    *n_out = v.size();
    if (v.size() > cap) return fail(PM_ECAP, "pm_counts_desc: %zu records needed, cap is %zu", v.size(), cap);
    for (size_t i = 0; i < v.size(); i++) {
        canonical_name(v[i]);
        out[i] = v[i];
    }
    return PM_OK;
}

extern "C" pm_status pm_counts_desc_interp(const char *description, const char *param, const pm_param *p, size_t np,
                                           int32_t *period, int32_t *degree) {
    if (!description || !param || !period || !degree || (np && !p)) return fail(PM_EINVAL, "pm_counts_desc_interp: NULL argument");
    Desc d;
    pm_status s = parse_desc(description, d);
    if (s) return s;
    std::vector<i64> pv(d.params.size(), 0);
    for (size_t i = 0; i < np; i++)
        for (size_t k = 0; k < d.params.size(); k++)
            if (p[i].key && d.params[k] == p[i].key) pv[k] = (i64)p[i].value;
    size_t P = 0;
    while (P < d.params.size() && d.params[P] != param) P++;
    if (P == d.params.size()) return fail(PM_EINVAL, "pm_counts_desc_interp: unknown parameter '%s'", param);
    i64 pe;
    int de;
    if ((s = derive_interp(d, (int)P, pv, &pe, &de))) return s;
    *period = (int32_t)pe;
    *degree = de;
    return PM_OK;
}
