// Model representation shared by pm_model.cpp (parsing, feature matching)
// and pm_fit.cu (GPU evaluation / calibration).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "pm.h"

namespace pm {

// SSA bytecode: instruction k computes value v[k] from earlier values.
enum OpCode : int32_t {
    OP_FEAT = 0,   // v = feature[arg]
    OP_PAR = 1,    // v = param[arg]
    OP_CONST = 2,  // v = c
    OP_ADD = 3,    // v = v[a] + v[b]
    OP_SUB = 4,
    OP_MUL = 5,
    OP_DIV = 6,
    OP_NEG = 7,    // v = -v[a]
    OP_TANH = 8,
    OP_EXP = 9,
    OP_LOG = 10,
    OP_SQRT = 11,
};

struct Ins {
    int32_t op;
    int32_t a, b;   // operand instruction indices
    int32_t arg;    // feature / parameter index
    double c;       // constant
};
static_assert(sizeof(Ins) == 24, "Ins layout");

constexpr int kMaxIns = 256;
constexpr int kMaxParamsFit = 16;

}  // namespace pm

struct pm_model {
    std::string out_feature, expr;
    std::vector<std::string> features, params;
    std::vector<pm::Ins> code;   // SSA program, last instruction is the result
    bool linear = false;         // g is homogeneous linear in the parameters
    std::vector<pm::Ins> start_code;  // same expression with tanh(.) -> 0 (start point)
    unsigned start_mask = 0;     // parameters that occur in start_code
    // device copy of `code` for the differentiation entry points (lazy)
    pm::Ins *d_code = nullptr;
    int d_device = -1;
    ~pm_model();
};
