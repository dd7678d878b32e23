// Model expressions (Section "Modeling Kernel Execution Time"): parsing to an
// SSA program, homogeneity analysis (is g linear in p?), and feature
// assembly -- matching model feature names against a kernel's feature
// records (Section "Data Motion Features": field order tag, memory type,
// data type, direction, lstrides, gstrides, afr; constraints such as >15).
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>

#include "pm_internal.h"
#include "pm_model.h"

namespace pm {
namespace {

struct Node {
    enum Kind { NUM, FEAT, PAR, NEG, ADD, SUB, MUL, DIV, FN } kind;
    double c = 0;
    std::string name;
    int fn = 0;  // OP_TANH.. for FN
    std::unique_ptr<Node> a, b;
};
typedef std::unique_ptr<Node> NP;

struct Parser {
    const char *s;
    size_t i = 0;
    std::string err;
    explicit Parser(const char *src) : s(src) {}
    void ws() {
        while (s[i] && isspace((unsigned char)s[i])) i++;
    }
    bool name_char(char ch) { return ch && !isspace((unsigned char)ch) && !strchr("+*/()", ch); }
    NP expr() {
        NP n = term();
        if (!n) return n;
        for (;;) {
            ws();
            char ch = s[i];
            if (ch != '+' && ch != '-') return n;
            i++;
            NP r = term();
            if (!r) return r;
            NP p(new Node{ch == '+' ? Node::ADD : Node::SUB});
            p->a = std::move(n);
            p->b = std::move(r);
            n = std::move(p);
        }
    }
    NP term() {
        NP n = unary();
        if (!n) return n;
        for (;;) {
            ws();
            char ch = s[i];
            if (ch != '*' && ch != '/') return n;
            i++;
            NP r = unary();
            if (!r) return r;
            NP p(new Node{ch == '*' ? Node::MUL : Node::DIV});
            p->a = std::move(n);
            p->b = std::move(r);
            n = std::move(p);
        }
    }
    NP unary() {
        ws();
        if (s[i] == '-') {
            i++;
            NP a = unary();
            if (!a) return a;
            NP p(new Node{Node::NEG});
            p->a = std::move(a);
            return p;
        }
        return prim();
    }
    NP prim() {
        ws();
        char ch = s[i];
        if (ch == '(') {
            i++;
            NP n = expr();
            if (!n) return n;
            ws();
            if (s[i] != ')') { err = "missing ')'"; return nullptr; }
            i++;
            return n;
        }
        if (isdigit((unsigned char)ch) || (ch == '.' && isdigit((unsigned char)s[i + 1]))) {
            char *end = nullptr;
            double v = strtod(s + i, &end);
            i = (size_t)(end - s);
            NP n(new Node{Node::NUM});
            n->c = v;
            return n;
        }
        if (isalpha((unsigned char)ch) || ch == '_') {
            size_t j = i;
            while (name_char(s[j])) j++;
            std::string nm(s + i, j - i);
            i = j;
            static const char *fns[4] = {"tanh", "exp", "log", "sqrt"};
            for (int k = 0; k < 4; k++)
                if (nm == fns[k]) {
                    ws();
                    if (s[i] != '(') { err = "expected '(' after " + nm; return nullptr; }
                    i++;
                    NP a = expr();
                    if (!a) return a;
                    ws();
                    if (s[i] != ')') { err = "missing ')'"; return nullptr; }
                    i++;
                    NP n(new Node{Node::FN});
                    n->fn = OP_TANH + k;
                    n->a = std::move(a);
                    return n;
                }
            if (nm.compare(0, 2, "f_") == 0) { NP n(new Node{Node::FEAT}); n->name = nm; return n; }
            if (nm.compare(0, 2, "p_") == 0) { NP n(new Node{Node::PAR}); n->name = nm; return n; }
            err = "unknown name '" + nm + "' (features start with f_, parameters with p_)";
            return nullptr;
        }
        err = ch ? std::string("unexpected '") + ch + "'" : "unexpected end of expression";
        return nullptr;
    }
};

int index_of(std::vector<std::string> &v, const std::string &s, bool add) {
    for (size_t k = 0; k < v.size(); k++)
        if (v[k] == s) return (int)k;
    if (!add) return -1;
    v.push_back(s);
    return (int)v.size() - 1;
}

void collect(const Node *n, pm_model *m) {
    if (!n) return;
    if (n->kind == Node::FEAT) index_of(m->features, n->name, true);
    if (n->kind == Node::PAR) index_of(m->params, n->name, true);
    collect(n->a.get(), m);
    collect(n->b.get(), m);
}

// Emit SSA; strip_tanh replaces every tanh(...) by the constant 0.
int emit(const Node *n, pm_model *m, std::vector<Ins> &code, bool strip_tanh) {
    Ins in{};
    switch (n->kind) {
    case Node::NUM: in.op = OP_CONST; in.c = n->c; break;
    case Node::FEAT: in.op = OP_FEAT; in.arg = index_of(m->features, n->name, false); break;
    case Node::PAR: in.op = OP_PAR; in.arg = index_of(m->params, n->name, false); break;
    case Node::NEG: in.op = OP_NEG; in.a = emit(n->a.get(), m, code, strip_tanh); break;
    case Node::FN:
        if (strip_tanh && n->fn == OP_TANH) { in.op = OP_CONST; in.c = 0.0; break; }
        in.op = n->fn;
        in.a = emit(n->a.get(), m, code, strip_tanh);
        break;
    default:
        in.op = n->kind == Node::ADD ? OP_ADD : n->kind == Node::SUB ? OP_SUB : n->kind == Node::MUL ? OP_MUL : OP_DIV;
        in.a = emit(n->a.get(), m, code, strip_tanh);
        in.b = emit(n->b.get(), m, code, strip_tanh);
    }
    // common subexpressions: reuse an identical earlier instruction
    for (size_t k = 0; k < code.size(); k++) {
        const Ins &o = code[k];
        if (o.op == in.op && o.a == in.a && o.b == in.b && o.arg == in.arg && memcmp(&o.c, &in.c, sizeof o.c) == 0)
            return (int)k;
    }
    code.push_back(in);
    return (int)code.size() - 1;
}

// Homogeneity class of an SSA program: 0 = parameter-free, 1 = homogeneous
// linear in the parameters, 2 = anything else.
int homog(const std::vector<Ins> &code) {
    std::vector<int> h(code.size());
    for (size_t k = 0; k < code.size(); k++) {
        const Ins &in = code[k];
        int x = 0;
        switch (in.op) {
        case OP_FEAT: case OP_CONST: x = 0; break;
        case OP_PAR: x = 1; break;
        case OP_ADD: case OP_SUB: {
            int a = h[in.a], b = h[in.b];
            x = (a == b && a < 2) ? a : 2;
            // a constant 0 (a stripped switch) keeps the other side's class
            if (a != b && a < 2 && b < 2) {
                if (code[in.a].op == OP_CONST && code[in.a].c == 0.0) x = b;
                else if (code[in.b].op == OP_CONST && code[in.b].c == 0.0) x = a;
            }
            break;
        }
        case OP_MUL: {
            int a = h[in.a], b = h[in.b];
            x = (a == 2 || b == 2 || a + b > 1) ? 2 : a + b;
            break;
        }
        case OP_DIV: x = h[in.b] == 0 ? h[in.a] : 2; break;
        case OP_NEG: x = h[in.a]; break;
        default: x = h[in.a] == 0 ? 0 : 2;
        }
        h[k] = x;
    }
    return h.back();
}

// ---------------------------------------------------------------- feature matching
struct Cons {
    int axis = -1;
    int cmp = 0;  // 0 =, 1 !=, 2 <, 3 >, 4 <=, 5 >=
    __int128 num = 0, den = 1;
};

bool parse_cons(const std::string &t, Cons &c) {
    size_t i = 0;
    if (t.compare(0, 2, "<=") == 0) { c.cmp = 4; i = 2; }
    else if (t.compare(0, 2, ">=") == 0) { c.cmp = 5; i = 2; }
    else if (t.compare(0, 2, "!=") == 0) { c.cmp = 1; i = 2; }
    else if (t[0] == '<') { c.cmp = 2; i = 1; }
    else if (t[0] == '>') { c.cmp = 3; i = 1; }
    else if (t[0] == '=') { c.cmp = 0; i = 1; }
    bool neg = false;
    if (i < t.size() && t[i] == '-') { neg = true; i++; }
    if (i >= t.size() || !isdigit((unsigned char)t[i])) return false;
    __int128 num = 0, den = 1;
    while (i < t.size() && isdigit((unsigned char)t[i])) num = num * 10 + (t[i++] - '0');
    if (i < t.size() && t[i] == '.') {
        i++;
        if (i >= t.size() || !isdigit((unsigned char)t[i])) return false;
        while (i < t.size() && isdigit((unsigned char)t[i])) { num = num * 10 + (t[i++] - '0'); den *= 10; }
    }
    if (i < t.size() && t[i] == '/') {
        i++;
        __int128 d = 0;
        if (i >= t.size()) return false;
        while (i < t.size() && isdigit((unsigned char)t[i])) d = d * 10 + (t[i++] - '0');
        if (d == 0) return false;
        den *= d;
    }
    if (i != t.size()) return false;
    c.num = neg ? -num : num;
    c.den = den;
    return true;
}

// x = xn / xd (xd > 0) against the constraint
bool cons_ok(const Cons &c, __int128 xn, __int128 xd) {
    __int128 l = xn * c.den, r = c.num * xd;
    switch (c.cmp) {
    case 0: return l == r;
    case 1: return l != r;
    case 2: return l < r;
    case 3: return l > r;
    case 4: return l <= r;
    default: return l >= r;
    }
}

struct Desc {
    int kind = -1;  // pm_feat_kind
    std::string dtype, op, tag;
    int mem = -1, dir = -1;
    std::vector<Cons> ls, gs;
    bool has_afr = false;
    Cons afr;
};

bool parse_strides(const std::string &body, std::vector<Cons> &out) {
    size_t i = 0;
    while (i < body.size()) {
        size_t j = body.find(';', i);
        if (j == std::string::npos) j = body.size();
        std::string part = body.substr(i, j - i);
        i = j + 1;
        if (part.empty()) continue;
        size_t colon = part.find(':');
        if (colon == std::string::npos || colon == 0) return false;
        for (size_t k = 0; k < colon; k++)
            if (!isdigit((unsigned char)part[k])) return false;
        Cons c;
        c.axis = atoi(part.substr(0, colon).c_str());
        if (c.axis > 2 || !parse_cons(part.substr(colon + 1), c)) return false;
        out.push_back(c);
    }
    return true;
}

bool is_dtype(const std::string &f) {
    return f == "float32" || f == "float64" || f == "float32x2" || f == "float32x4" || f == "float64x2" ||
           f == "bfloat16" || f == "tfloat32";
}

pm_status parse_desc(const std::string &name, Desc &d) {
    if (name == "f_sync_barrier_local") { d.kind = PM_FEAT_SYNC; return PM_OK; }
    if (name == "f_thread_groups") { d.kind = PM_FEAT_GROUPS; return PM_OK; }
    if (name == "f_sync_kernel_launch") { d.kind = PM_FEAT_LAUNCH; return PM_OK; }
    if (name.compare(0, 5, "f_op_") == 0) {
        std::string rest = name.substr(5);
        size_t u = rest.find('_');
        if (u == std::string::npos) return fail(PM_EPARSE, "bad op feature '%s'", name.c_str());
        d.kind = PM_FEAT_OP;
        d.dtype = rest.substr(0, u);
        d.op = rest.substr(u + 1);
        if (!is_dtype(d.dtype) || (d.op != "add" && d.op != "mul" && d.op != "madd"))
            return fail(PM_EPARSE, "bad op feature '%s'", name.c_str());
        return PM_OK;
    }
    if (name.compare(0, 12, "f_mem_access") == 0) {
        d.kind = PM_FEAT_MEM;
        std::string rest = name.substr(12);
        int pos = 0;  // field order: tag 0, mem 1, dtype 2, dir 3, lstrides 4, gstrides 5, afr 6
        size_t i = 0;
        while (i < rest.size()) {
            size_t j = rest.find('_', i);
            if (j == std::string::npos) j = rest.size();
            std::string f = rest.substr(i, j - i);
            i = j + 1;
            if (f.empty()) continue;
            int k;
            if (f.compare(0, 4, "tag:") == 0) { k = 0; d.tag = f.substr(4); }
            else if (f == "global" || f == "local") { k = 1; d.mem = f == "local"; }
            else if (is_dtype(f)) { k = 2; d.dtype = f; }
            else if (f == "load" || f == "store") { k = 3; d.dir = f == "store"; }
            else if (f.compare(0, 10, "lstrides:{") == 0 && f.back() == '}') {
                k = 4;
                if (!parse_strides(f.substr(10, f.size() - 11), d.ls))
                    return fail(PM_EPARSE, "bad lstrides in '%s'", name.c_str());
            } else if (f.compare(0, 10, "gstrides:{") == 0 && f.back() == '}') {
                k = 5;
                if (!parse_strides(f.substr(10, f.size() - 11), d.gs))
                    return fail(PM_EPARSE, "bad gstrides in '%s'", name.c_str());
            } else if (f.compare(0, 4, "afr:") == 0) {
                k = 6;
                d.has_afr = true;
                if (!parse_cons(f.substr(4), d.afr)) return fail(PM_EPARSE, "bad afr in '%s'", name.c_str());
            } else
                return fail(PM_EPARSE, "bad field '%s' in '%s'", f.c_str(), name.c_str());
            if (k < pos) return fail(PM_EPARSE, "field '%s' out of order in '%s'", f.c_str(), name.c_str());
            pos = k + 1;
        }
        return PM_OK;
    }
    return fail(PM_EPARSE, "unknown feature '%s'", name.c_str());
}

bool desc_match(const Desc &d, const pm_feature &f) {
    if (d.kind != f.kind) return false;
    if (d.kind == PM_FEAT_OP) return d.dtype == f.dtype && d.op == f.op;
    if (d.kind != PM_FEAT_MEM) return true;
    if (!d.tag.empty() && d.tag != f.tag) return false;
    if (d.mem >= 0 && d.mem != f.mem) return false;
    if (!d.dtype.empty() && d.dtype != f.dtype) return false;
    if (d.dir >= 0 && d.dir != f.dir) return false;
    for (const Cons &c : d.ls)
        if (c.axis >= f.nl || !cons_ok(c, f.lstride[c.axis], 1)) return false;
    for (const Cons &c : d.gs)
        if (c.axis >= f.ng || !cons_ok(c, f.gstride[c.axis], 1)) return false;
    if (d.has_afr && (f.footprint == 0 || !cons_ok(d.afr, (__int128)f.accesses, (__int128)f.footprint))) return false;
    return true;
}

}  // namespace
}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_model_create(const char *out_feature, const char *expr, pm_model **m) {
    if (!out_feature || !expr || !m) return fail(PM_EINVAL, "pm_model_create: NULL argument");
    Parser p(expr);
    NP root = p.expr();
    if (!root) return fail(PM_EPARSE, "model expression: %s at offset %zu", p.err.c_str(), p.i);
    p.ws();
    if (expr[p.i]) return fail(PM_EPARSE, "model expression: trailing input at offset %zu", p.i);
    pm_model *mm = new (std::nothrow) pm_model();
    if (!mm) return fail(PM_ENOMEM, "pm_model_create: out of memory");
    mm->out_feature = out_feature;
    mm->expr = expr;
    collect(root.get(), mm);
    emit(root.get(), mm, mm->code, false);
    emit(root.get(), mm, mm->start_code, true);
    if (mm->code.size() > (size_t)kMaxIns || mm->params.size() > (size_t)kMaxParamsFit || mm->params.empty()) {
        delete mm;
        return fail(PM_EPARSE, "model: need 1..%d parameters and <= %d operations", kMaxParamsFit, kMaxIns);
    }
    for (auto &f : mm->features) {
        Desc d;
        if (parse_desc(f, d)) {
            delete mm;
            return PM_EPARSE;
        }
    }
    mm->linear = homog(mm->code) == 1;
    for (const Ins &in : mm->start_code)
        if (in.op == OP_PAR) mm->start_mask |= 1u << in.arg;
    *m = mm;
    return PM_OK;
}

void pm_model_destroy(pm_model *m) { delete m; }

pm_status pm_model_info(const pm_model *m, size_t *nf, size_t *np) {
    if (!m) return fail(PM_EINVAL, "pm_model_info: NULL model");
    if (nf) *nf = m->features.size();
    if (np) *np = m->params.size();
    return PM_OK;
}

pm_status pm_model_feature_name(const pm_model *m, size_t i, const char **name) {
    if (!m || !name || i >= m->features.size()) return fail(PM_EINVAL, "pm_model_feature_name: bad argument");
    *name = m->features[i].c_str();
    return PM_OK;
}

pm_status pm_model_param_name(const pm_model *m, size_t i, const char **name) {
    if (!m || !name || i >= m->params.size()) return fail(PM_EINVAL, "pm_model_param_name: bad argument");
    *name = m->params[i].c_str();
    return PM_OK;
}

pm_status pm_model_is_linear(const pm_model *m, int32_t *linear) {
    if (!m || !linear) return fail(PM_EINVAL, "pm_model_is_linear: NULL argument");
    *linear = m->linear ? 1 : 0;
    return PM_OK;
}

pm_status pm_feature_values(const pm_model *m, const pm_feature *feats, size_t nfeat, double *row_out) {
    if (!m || !row_out || (nfeat && !feats)) return fail(PM_EINVAL, "pm_feature_values: NULL argument");
    for (size_t k = 0; k < m->features.size(); k++) {
        Desc d;
        pm_status s = parse_desc(m->features[k], d);
        if (s) return s;
        unsigned long long sum = 0;
        for (size_t r = 0; r < nfeat; r++)
            if (desc_match(d, feats[r])) sum += feats[r].count;
        row_out[k] = (double)sum;
    }
    return PM_OK;
}

}  // extern "C"
