// kl_def.cpp -- user-defined tunable kernels: the kernel definition of
// Sec. 4.1 for any CUDA kernel, with the same capture (Sec. 4.2), tuning
// (Sec. 4.3), wisdom (Sec. 4.4) and run-time selection and compilation
// (Sec. 4.5) as the built-in stencil.
//
// A definition holds the kernel's source text and function name, its
// tunable parameters (each a list of integer values and a default, passed to
// NVRTC as -D<name>=<value>), restrictions (integer expressions over the
// parameters that must be non-zero) and the launch geometry (block size,
// grid size and dynamic shared memory as integer expressions over the
// parameters and the problem size problem_x, problem_y, problem_z).

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <fstream>
#include <functional>
#include <future>
#include <memory>
#include <random>
#include <set>
#include <sstream>
#include <thread>

#include "kl_internal.h"

namespace kl {
namespace {

// ============================================================ expressions
//
// Integer expressions in C syntax: literals, names, unary - ! ~, binary
// * / % + - < <= > >= == != & ^ | && ||, the conditional a ? b : c, and the
// functions min(a, b), max(a, b), div_ceil(a, b) and round_up(a, b) (a
// rounded up to a multiple of b).  Evaluation is in 64-bit integers; division
// or remainder by zero and overflow are errors.

struct Expr {
    enum Kind { Num, Var, Unary, Binary, Cond, Call } kind = Num;
    int64_t num = 0;
    std::string name;                    // variable, operator or function
    std::vector<std::shared_ptr<Expr>> kids;
};
using ExprP = std::shared_ptr<Expr>;

class Parser {
  public:
    explicit Parser(const std::string &s) : s_(s) {}

    ExprP parse(std::string *err)
    {
        ExprP e = cond();
        skip();
        if (e && p_ != s_.size()) fail_at("unexpected '" + s_.substr(p_, 1) + "'");
        if (!err_.empty()) {
            *err = err_;
            return nullptr;
        }
        return e;
    }

  private:
    const std::string &s_;
    size_t p_ = 0;
    std::string err_;

    void fail_at(const std::string &m)
    {
        if (err_.empty()) err_ = m + " at offset " + std::to_string(p_) + " of \"" + s_ + "\"";
    }
    void skip()
    {
        while (p_ < s_.size() && isspace((unsigned char)s_[p_])) ++p_;
    }
    bool eat(const char *op)
    {
        skip();
        size_t n = strlen(op);
        if (s_.compare(p_, n, op) != 0) return false;
        // do not take the first character of a longer operator
        if (n == 1 && p_ + 1 < s_.size()) {
            char a = s_[p_], b = s_[p_ + 1];
            if ((a == '<' || a == '>' || a == '=' || a == '!') && b == '=') return false;
            if ((a == '&' && b == '&') || (a == '|' && b == '|')) return false;
        }
        p_ += n;
        return true;
    }
    static ExprP node(Expr::Kind k, const std::string &name, std::vector<ExprP> kids)
    {
        auto e = std::make_shared<Expr>();
        e->kind = k;
        e->name = name;
        e->kids = std::move(kids);
        return e;
    }
    ExprP cond()
    {
        ExprP c = binary(0);
        if (!c) return nullptr;
        if (eat("?")) {
            ExprP a = cond();
            if (!a) return nullptr;
            if (!eat(":")) {
                fail_at("expected ':'");
                return nullptr;
            }
            ExprP b = cond();
            if (!b) return nullptr;
            return node(Expr::Cond, "?", {c, a, b});
        }
        return c;
    }
    // precedence levels, loosest first
    ExprP binary(int level)
    {
        static const std::vector<std::vector<const char *>> ops = {
            {"||"}, {"&&"}, {"|"}, {"^"}, {"&"}, {"==", "!="}, {"<=", ">=", "<", ">"},
            {"+", "-"}, {"*", "/", "%"}};
        if (level == (int)ops.size()) return unary();
        ExprP a = binary(level + 1);
        while (a) {
            const char *hit = nullptr;
            for (const char *op : ops[level])
                if (eat(op)) {
                    hit = op;
                    break;
                }
            if (!hit) break;
            ExprP b = binary(level + 1);
            if (!b) return nullptr;
            a = node(Expr::Binary, hit, {a, b});
        }
        return a;
    }
    ExprP unary()
    {
        for (const char *op : {"-", "!", "~", "+"})
            if (eat(op)) {
                ExprP a = unary();
                if (!a) return nullptr;
                return node(Expr::Unary, op, {a});
            }
        return primary();
    }
    ExprP primary()
    {
        skip();
        if (p_ >= s_.size()) {
            fail_at("unexpected end");
            return nullptr;
        }
        char c = s_[p_];
        if (c == '(') {
            ++p_;
            ExprP e = cond();
            if (!e) return nullptr;
            if (!eat(")")) {
                fail_at("expected ')'");
                return nullptr;
            }
            return e;
        }
        if (isdigit((unsigned char)c)) {
            size_t q = p_;
            int64_t v = 0;
            while (q < s_.size() && isdigit((unsigned char)s_[q])) {
                if (__builtin_mul_overflow(v, (int64_t)10, &v) ||
                    __builtin_add_overflow(v, (int64_t)(s_[q] - '0'), &v)) {
                    fail_at("literal too large");
                    return nullptr;
                }
                ++q;
            }
            p_ = q;
            auto e = std::make_shared<Expr>();
            e->kind = Expr::Num;
            e->num = v;
            return e;
        }
        if (isalpha((unsigned char)c) || c == '_') {
            size_t q = p_;
            while (q < s_.size() && (isalnum((unsigned char)s_[q]) || s_[q] == '_')) ++q;
            std::string id = s_.substr(p_, q - p_);
            p_ = q;
            if (eat("(")) {
                std::vector<ExprP> args;
                if (!eat(")")) {
                    do {
                        ExprP a = cond();
                        if (!a) return nullptr;
                        args.push_back(a);
                    } while (eat(","));
                    if (!eat(")")) {
                        fail_at("expected ')' after arguments");
                        return nullptr;
                    }
                }
                if ((id != "min" && id != "max" && id != "div_ceil" && id != "round_up") ||
                    args.size() != 2) {
                    fail_at("unknown function " + id + " (min, max, div_ceil, round_up take two arguments)");
                    return nullptr;
                }
                return node(Expr::Call, id, args);
            }
            return node(Expr::Var, id, {});
        }
        fail_at(std::string("unexpected '") + c + "'");
        return nullptr;
    }
};

using Lookup = std::function<bool(const std::string &, int64_t *)>;

bool eval(const Expr &e, const Lookup &var, int64_t *out, std::string *err)
{
    int64_t a = 0, b = 0, c = 0;
    switch (e.kind) {
    case Expr::Num:
        *out = e.num;
        return true;
    case Expr::Var:
        if (!var(e.name, out)) {
            *err = "unknown name '" + e.name + "'";
            return false;
        }
        return true;
    case Expr::Unary:
        if (!eval(*e.kids[0], var, &a, err)) return false;
        if (e.name == "-") {
            if (a == INT64_MIN) {
                *err = "overflow";
                return false;
            }
            *out = -a;
        } else if (e.name == "!") {
            *out = !a;
        } else if (e.name == "~") {
            *out = ~a;
        } else {
            *out = a;
        }
        return true;
    case Expr::Cond:
        if (!eval(*e.kids[0], var, &c, err)) return false;
        return eval(*e.kids[c ? 1 : 2], var, out, err);
    case Expr::Binary: {
        const std::string &op = e.name;
        if (!eval(*e.kids[0], var, &a, err)) return false;
        if (op == "&&" && !a) return *out = 0, true;
        if (op == "||" && a) return *out = 1, true;
        if (!eval(*e.kids[1], var, &b, err)) return false;
        bool ovf = false;
        if (op == "+") ovf = __builtin_add_overflow(a, b, out);
        else if (op == "-") ovf = __builtin_sub_overflow(a, b, out);
        else if (op == "*") ovf = __builtin_mul_overflow(a, b, out);
        else if (op == "/" || op == "%") {
            if (b == 0) {
                *err = "division by zero";
                return false;
            }
            if (a == INT64_MIN && b == -1) ovf = true;
            else *out = op == "/" ? a / b : a % b;
        } else if (op == "<") *out = a < b;
        else if (op == "<=") *out = a <= b;
        else if (op == ">") *out = a > b;
        else if (op == ">=") *out = a >= b;
        else if (op == "==") *out = a == b;
        else if (op == "!=") *out = a != b;
        else if (op == "&") *out = a & b;
        else if (op == "^") *out = a ^ b;
        else if (op == "|") *out = a | b;
        else if (op == "&&" || op == "||") *out = b != 0;
        if (ovf) {
            *err = "overflow";
            return false;
        }
        return true;
    }
    case Expr::Call:
        if (!eval(*e.kids[0], var, &a, err) || !eval(*e.kids[1], var, &b, err)) return false;
        if (e.name == "min") *out = std::min(a, b);
        else if (e.name == "max") *out = std::max(a, b);
        else {
            if (b <= 0) {
                *err = e.name + ": the divisor must be positive";
                return false;
            }
            int64_t q = a / b + ((a % b) > 0 ? 1 : 0);
            if (e.name == "div_ceil") *out = q;
            else if (__builtin_mul_overflow(q, b, out)) {
                *err = "overflow";
                return false;
            }
        }
        return true;
    }
    return false;
}

void names_of(const Expr &e, std::set<std::string> *out)
{
    if (e.kind == Expr::Var) out->insert(e.name);
    for (auto &k : e.kids) names_of(*k, out);
}

bool valid_ident(const std::string &s)
{
    if (s.empty() || !(isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
    for (char c : s)
        if (!(isalnum((unsigned char)c) || c == '_')) return false;
    return true;
}

}  // namespace

}  // namespace kl

struct kl_def {
    std::string name, source, function, options;
    struct Param {
        std::string name;
        std::vector<int64_t> values;
        int64_t dflt = 0;
    };
    std::vector<Param> params;
    std::vector<std::pair<std::string, kl::ExprP>> restrictions;
    std::string geo_text[7];    // block x, y, z, grid x, y, z, shared memory
    kl::ExprP geo[7];
    std::map<std::string, std::string> selection;   // context + problem -> configuration text
    std::string last_config;
    int last_rule = 0;
};

namespace kl {

using Values = std::vector<int64_t>;

static const char *kGeoNames[7] = {"block_x", "block_y", "block_z", "grid_x", "grid_y", "grid_z",
                                   "shared_memory"};

static std::string config_text(const kl_def &d, const Values &v)
{
    std::string s;
    for (size_t q = 0; q < d.params.size(); ++q)
        s += (q ? "," : "") + d.params[q].name + "=" + std::to_string(v[q]);
    return s.empty() ? "default" : s;
}

static Values default_values(const kl_def &d)
{
    Values v;
    for (auto &p : d.params) v.push_back(p.dflt);
    return v;
}

// "default", or name=value pairs separated by commas; unnamed parameters keep
// their defaults; every value must be one of the parameter's values
static bool parse_config(const kl_def &d, const std::string &text, Values *v, std::string *err)
{
    *v = default_values(d);
    if (text.empty() || text == "default") return true;
    std::stringstream ss(text);
    std::string item;
    std::set<std::string> seen;
    while (std::getline(ss, item, ',')) {
        size_t eq = item.find('=');
        if (eq == std::string::npos) {
            *err = "configuration item without '=': " + item;
            return false;
        }
        std::string k = item.substr(0, eq), val = item.substr(eq + 1);
        size_t q = 0;
        while (q < d.params.size() && d.params[q].name != k) ++q;
        if (q == d.params.size()) {
            *err = "unknown parameter '" + k + "'";
            return false;
        }
        if (!seen.insert(k).second) {
            *err = "parameter '" + k + "' given twice";
            return false;
        }
        char *end = nullptr;
        long long x = strtoll(val.c_str(), &end, 10);
        if (val.empty() || *end) {
            *err = "value of '" + k + "' is not an integer: " + val;
            return false;
        }
        auto &vals = d.params[q].values;
        if (std::find(vals.begin(), vals.end(), (int64_t)x) == vals.end()) {
            *err = "value " + val + " is not one of the values of '" + k + "'";
            return false;
        }
        (*v)[q] = x;
    }
    return true;
}

static int64_t raw_size(const kl_def &d)
{
    int64_t n = 1;
    for (auto &p : d.params) {
        if (n > INT64_MAX / (int64_t)p.values.size()) return -1;
        n *= (int64_t)p.values.size();
    }
    return n;
}

// the idx-th point of the raw space (first parameter varies fastest)
static Values values_at(const kl_def &d, int64_t idx)
{
    Values v;
    for (auto &p : d.params) {
        int64_t r = (int64_t)p.values.size();
        v.push_back(p.values[(size_t)(idx % r)]);
        idx /= r;
    }
    return v;
}

static bool restrictions_hold(const kl_def &d, const Values &v, std::string *err)
{
    Lookup look = [&](const std::string &n, int64_t *out) {
        for (size_t q = 0; q < d.params.size(); ++q)
            if (d.params[q].name == n) {
                *out = v[q];
                return true;
            }
        return false;
    };
    for (auto &r : d.restrictions) {
        int64_t x = 0;
        if (!eval(*r.second, look, &x, err)) {
            *err = "restriction \"" + r.first + "\": " + *err;
            return false;
        }
        if (!x) {
            *err = "restriction \"" + r.first + "\" does not hold";
            return false;
        }
    }
    return true;
}

// block, grid and shared memory of a configuration for a problem
static bool geometry(const kl_def &d, const Values &v, const int64_t problem[3], int64_t out[7],
                     std::string *err)
{
    Lookup look = [&](const std::string &n, int64_t *o) {
        for (size_t q = 0; q < d.params.size(); ++q)
            if (d.params[q].name == n) {
                *o = v[q];
                return true;
            }
        if (n == "problem_x") return *o = problem[0], true;
        if (n == "problem_y") return *o = problem[1], true;
        if (n == "problem_z") return *o = problem[2], true;
        return false;
    };
    for (int q = 0; q < 7; ++q) {
        if (!d.geo[q]) {
            // defaults: block 1, grid = div_ceil(problem, block), no shared memory
            out[q] = q < 3 ? 1 : q < 6 ? (problem[q - 3] + out[q - 3] - 1) / out[q - 3] : 0;
            continue;
        }
        if (!eval(*d.geo[q], look, &out[q], err)) {
            *err = std::string(kGeoNames[q]) + ": " + *err;
            return false;
        }
    }
    for (int q = 0; q < 3; ++q)
        if (out[q] < 1 || out[q + 3] < 1) {
            *err = std::string(kGeoNames[out[q] < 1 ? q : q + 3]) + " is below 1";
            return false;
        }
    if (out[0] > 1024 || out[1] > 1024 || out[2] > 64 || out[0] * out[1] * out[2] > 1024) {
        *err = "more than 1024 threads per block (or a block dimension above its limit)";
        return false;
    }
    if (out[3] > 2147483647LL || out[4] > 65535 || out[5] > 65535) {
        *err = "grid dimension above its limit";
        return false;
    }
    if (out[6] < 0 || out[6] > 232448) {
        *err = "dynamic shared memory outside 0..227 KB";
        return false;
    }
    return true;
}

static uint64_t def_hash(const kl_def &d)
{
    std::string s = d.name + '\0' + d.function + '\0' + d.options + '\0' + d.source;
    return fnv1a(s.data(), s.size());
}

static std::string def_defines(const kl_def &d, const Values &v)
{
    std::string s;
    for (size_t q = 0; q < d.params.size(); ++q)
        s += " -D" + d.params[q].name + "=" + std::to_string(v[q]);
    return s + (d.options.empty() ? "" : " " + d.options);
}

static kl_status def_compile(const kl_def &d, const std::string &defines, bool verbose, Compiled *out)
{
    nvrtcProgram prog;
    std::string fname = "kl_def_" + d.name + ".cu";
    nvrtcResult r = nvrtcCreateProgram(&prog, d.source.c_str(), fname.c_str(), 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS) return fail(KL_ERR_NVRTC, nvrtcGetErrorString(r));
    r = nvrtcAddNameExpression(prog, d.function.c_str());
    std::vector<std::string> opts = {"-arch=sm_103a", "-std=c++17", "-lineinfo"};
    if (verbose) opts.push_back("--ptxas-options=-v");
    std::stringstream ss(defines);
    std::string tok;
    while (ss >> tok) opts.push_back(tok);
    std::vector<const char *> cops;
    for (auto &o : opts) cops.push_back(o.c_str());
    if (r == NVRTC_SUCCESS) r = nvrtcCompileProgram(prog, (int)cops.size(), cops.data());
    size_t logn = 0;
    nvrtcGetProgramLogSize(prog, &logn);
    out->log.assign(logn, '\0');
    if (logn) nvrtcGetProgramLog(prog, &out->log[0]);
    while (!out->log.empty() && out->log.back() == '\0') out->log.pop_back();
    const char *lowered = nullptr;
    if (r == NVRTC_SUCCESS) r = nvrtcGetLoweredName(prog, d.function.c_str(), &lowered);
    if (r != NVRTC_SUCCESS) {
        nvrtcDestroyProgram(&prog);
        return fail(KL_ERR_NVRTC, std::string("NVRTC (") + d.name + "): " + nvrtcGetErrorString(r) +
                                      "\n" + defines + "\n" + out->log);
    }
    out->symbol = lowered;
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    out->cubin.resize(n);
    nvrtcGetCUBIN(prog, out->cubin.data());
    nvrtcDestroyProgram(&prog);
    return KL_OK;
}

static kl_status def_load(kl_ctx *ctx, const std::string &key, const Compiled &c, DefKernel **out)
{
    DefKernel k;
    CUresult r = ctx->drv.ModuleLoadData(&k.mod, c.cubin.data());
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuModuleLoadData (user kernel)");
    r = ctx->drv.ModuleGetFunction(&k.fn, k.mod, c.symbol.c_str());
    if (r != CUDA_SUCCESS) {
        ctx->drv.ModuleUnload(k.mod);
        return cu_fail(r, "cuModuleGetFunction (user kernel)");
    }
    auto ins = ctx->def_kernels.emplace(key, k);
    *out = &ins.first->second;
    return KL_OK;
}

// compiled function of one configuration: context memory, disk cache, NVRTC
static kl_status def_kernel(kl_ctx *ctx, const kl_def &d, const Values &v, DefKernel **out)
{
    std::string defines = def_defines(d, v);
    std::string ident = cache_identity(def_hash(d), defines);
    auto it = ctx->def_kernels.find(ident);
    if (it != ctx->def_kernels.end()) {
        ctx->cache_hits++;
        *out = &it->second;
        return KL_OK;
    }
    auto t0 = std::chrono::steady_clock::now();
    auto ms = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    Compiled c;
    if (!ctx->cache_dir.empty() && cache_read(ctx->cache_dir, ident, &c)) {
        ctx->t_disk_ms += ms();
        if (def_load(ctx, ident, c, out) == KL_OK) {
            ctx->disk_hits++;
            ctx->cache_misses++;
            return KL_OK;
        }
        cudaGetLastError();
        t0 = std::chrono::steady_clock::now();
    }
    kl_status st = def_compile(d, defines, false, &c);
    if (st) return st;
    ctx->t_nvrtc_ms += ms();
    if (!ctx->cache_dir.empty() && cache_write(ctx->cache_dir, ident, c)) ctx->disk_writes++;
    ctx->cache_misses++;
    return def_load(ctx, ident, c, out);
}

static kl_status check_args(int32_t nargs, const kl_arg *args)
{
    if (nargs < 0 || nargs > 64 || (nargs > 0 && !args))
        return fail(KL_ERR_INVALID_ARG, "arguments: need 0..64 and a non-NULL array");
    for (int q = 0; q < nargs; ++q) {
        const kl_arg &a = args[q];
        if (a.kind < 0 || a.kind > 3)
            return fail(KL_ERR_INVALID_ARG, "argument " + std::to_string(q) + ": kind must be 0..3");
        if (a.kind == 0 && (!a.ptr || a.bytes < 1 || a.bytes > 64))
            return fail(KL_ERR_INVALID_ARG, "argument " + std::to_string(q) +
                                                ": a scalar needs a value pointer and 1..64 bytes");
        if (a.kind > 0 && (a.bytes < 0 || (a.bytes > 0 && !a.ptr)))
            return fail(KL_ERR_INVALID_ARG, "argument " + std::to_string(q) + ": bad buffer");
        if (a.kind > 0 && (a.dtype < 0 || a.dtype > 5))
            return fail(KL_ERR_INVALID_ARG, "argument " + std::to_string(q) + ": dtype must be 0..5");
    }
    return KL_OK;
}

static kl_status def_launch_values(kl_ctx *ctx, kl_def *d, const Values &v, const int64_t problem[3],
                                   int32_t nargs, const kl_arg *args, cudaStream_t s)
{
    std::string err;
    if (!restrictions_hold(*d, v, &err)) return fail(KL_ERR_INVALID_ARG, config_text(*d, v) + ": " + err);
    int64_t geo[7];
    if (!geometry(*d, v, problem, geo, &err)) return fail(KL_ERR_INVALID_ARG, config_text(*d, v) + ": " + err);
    DefKernel *k = nullptr;
    kl_status st = def_kernel(ctx, *d, v, &k);
    if (st) return st;
    if (geo[6] > k->smem_attr) {
        CUresult r = ctx->drv.FuncSetAttribute(k->fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                               (int)geo[6]);
        if (r != CUDA_SUCCESS) return cu_fail(r, "cuFuncSetAttribute (user kernel shared memory)");
        k->smem_attr = (int)geo[6];
    }
    std::vector<const void *> dptr((size_t)nargs);
    std::vector<void *> kp((size_t)nargs);
    for (int q = 0; q < nargs; ++q) {
        if (args[q].kind == 0) {
            kp[q] = const_cast<void *>(args[q].ptr);
        } else {
            dptr[q] = args[q].ptr;
            kp[q] = &dptr[q];
        }
    }
    CUresult r = ctx->drv.LaunchKernel(k->fn, (unsigned)geo[3], (unsigned)geo[4], (unsigned)geo[5],
                                       (unsigned)geo[0], (unsigned)geo[1], (unsigned)geo[2],
                                       (unsigned)geo[6], (CUstream)s, nargs ? kp.data() : nullptr,
                                       nullptr);
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuLaunchKernel (user kernel)");
    ctx->launches++;
    d->last_config = config_text(*d, v);
    return KL_OK;
}

// a problem extent as the 32-bit size of a wisdom record (nearest-size
// selection only needs the magnitude)
static int wisdom_extent(int64_t x)
{
    return (int)std::max<int64_t>(0, std::min<int64_t>(x, 2147483647));
}

static std::string def_wisdom_path(const kl_ctx *ctx, const kl_def &d)
{
    return (ctx->wisdom_dir.empty() ? std::string(".") : ctx->wisdom_dir) + "/" + d.name + ".wisdom";
}

// ------------------------------------------------------------- capture

struct DefCapture {
    std::string name, function;
    int64_t problem[3] = {0, 0, 0};
    std::vector<kl_arg> args;                 // ptr unused
    std::vector<std::vector<char>> data;      // scalar value or buffer contents (inputs)
};

static kl_status def_capture_read(const std::string &path, DefCapture *c)
{
    FILE *f = fopen(path.c_str(), "rb");
    if (!f) return fail(KL_ERR_IO, "cannot open capture " + path);
    char line[8192];
    int nargs = -1;
    bool ok = fgets(line, sizeof line, f) && strncmp(line, "KLDEFCAP1", 9) == 0, end = false;
    auto rest = [&](const char *key) -> std::string {
        std::string s = line + strlen(key);
        while (!s.empty() && (s.back() == '\n' || s.back() == '\r')) s.pop_back();
        return s;
    };
    while (ok && fgets(line, sizeof line, f)) {
        long long px, py, pz, bytes;
        int q, kind, dtype;
        if (strncmp(line, "END", 3) == 0) {
            end = true;
            break;
        } else if (strncmp(line, "name ", 5) == 0) {
            c->name = rest("name ");
        } else if (strncmp(line, "function ", 9) == 0) {
            c->function = rest("function ");
        } else if (sscanf(line, "problem %lld %lld %lld", &px, &py, &pz) == 3) {
            c->problem[0] = px;
            c->problem[1] = py;
            c->problem[2] = pz;
        } else if (sscanf(line, "nargs %d", &nargs) == 1) {
        } else if (sscanf(line, "arg %d %d %lld %d", &q, &kind, &bytes, &dtype) == 4) {
            if (q != (int)c->args.size() || bytes < 0 || kind < 0 || kind > 3) ok = false;
            kl_arg a{nullptr, bytes, kind, dtype};
            c->args.push_back(a);
        }
    }
    if (!ok || !end || nargs < 0 || nargs != (int)c->args.size() || c->name.empty()) {
        fclose(f);
        return fail(KL_ERR_WISDOM_PARSE, "capture: malformed header in " + path);
    }
    for (auto &a : c->args) {
        std::vector<char> b(a.kind == 2 ? 0 : (size_t)a.bytes);
        if (!b.empty() && fread(b.data(), 1, b.size(), f) != b.size()) {
            fclose(f);
            return fail(KL_ERR_WISDOM_PARSE, "capture: truncated data in " + path);
        }
        c->data.push_back(std::move(b));
    }
    fclose(f);
    return KL_OK;
}

// ---------------------------------------------------------------- tuning

struct DefOpts {
    std::string strategy = "random", log;
    double budget_s = 60, verify_tol = -1;
    int max_evals = 100, reps = 7, warm = 2, threads = 0;
    unsigned seed = 1;
};

static kl_status def_parse_opts(const char *text, DefOpts *o)
{
    if (!text) return KL_OK;
    std::stringstream ss(text);
    std::string tok;
    while (ss >> tok) {
        size_t eq = tok.find('=');
        if (eq == std::string::npos) return fail(KL_ERR_INVALID_ARG, "tune option without '=': " + tok);
        std::string k = tok.substr(0, eq), v = tok.substr(eq + 1);
        if (k == "strategy") o->strategy = v;
        else if (k == "budget_s") o->budget_s = atof(v.c_str());
        else if (k == "max_evals") o->max_evals = atoi(v.c_str());
        else if (k == "seed") o->seed = (unsigned)strtoul(v.c_str(), nullptr, 10);
        else if (k == "verify_tol") o->verify_tol = atof(v.c_str());
        else if (k == "log") o->log = v;
        else if (k == "reps") o->reps = std::max(1, atoi(v.c_str()));
        else if (k == "warm") o->warm = std::max(0, atoi(v.c_str()));
        else if (k == "threads") o->threads = atoi(v.c_str());
        else return fail(KL_ERR_INVALID_ARG, "unknown tune option '" + k + "'");
    }
    if (o->strategy != "random" && o->strategy != "exhaustive" && o->strategy != "bayes")
        return fail(KL_ERR_INVALID_ARG, "strategy must be random, exhaustive or bayes");
    return KL_OK;
}

// value of element i of a buffer of dtype 0..3 (f64, f32, bf16, f16)
static double element(int32_t dtype, const std::vector<char> &a, size_t i)
{
    if (dtype == 0) {
        double x;
        memcpy(&x, &a[8 * i], 8);
        return x;
    }
    if (dtype == 1) {
        float x;
        memcpy(&x, &a[4 * i], 4);
        return x;
    }
    uint16_t h;
    memcpy(&h, &a[2 * i], 2);
    if (dtype == 2) {                       // bfloat16: the upper half of an f32
        uint32_t u = (uint32_t)h << 16;
        float x;
        memcpy(&x, &u, 4);
        return x;
    }
    // IEEE binary16: sign, 5-bit exponent (bias 15), 10-bit fraction
    int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
    double v = e == 0 ? std::ldexp((double)m, -24)
               : e == 31 ? (m ? NAN : INFINITY)
                         : std::ldexp((double)(m | 1024), e - 25);
    return s ? -v : v;
}

// largest |a - b| over max |b| for floating types (NaN on one side only:
// infinite), else the number of differing bytes
static double compare(int32_t dtype, const std::vector<char> &a, const std::vector<char> &b)
{
    if (dtype <= 3) {
        size_t n = a.size() / (dtype == 0 ? 8 : dtype == 1 ? 4 : 2);
        double d = 0, m = 0;
        for (size_t i = 0; i < n; ++i) {
            double x = element(dtype, a, i), y = element(dtype, b, i);
            if (std::isnan(x) != std::isnan(y)) return INFINITY;
            if (!std::isnan(x)) {
                d = std::max(d, std::fabs(x - y));
                m = std::max(m, std::fabs(y));
            }
        }
        return m > 0 ? d / m : d;
    }
    size_t diff = 0;
    for (size_t i = 0; i < a.size(); ++i) diff += a[i] != b[i];
    return (double)diff;
}

// default verification tolerance of an output of dtype
static double default_tol(int32_t dtype)
{
    return dtype == 0 ? 1e-12 : dtype == 1 ? 1e-5 : dtype <= 3 ? 1e-2 : 0.0;
}

}  // namespace kl

using namespace kl;

void kl::def_kernels_unload(kl_ctx *ctx)
{
    for (auto &p : ctx->def_kernels)
        if (p.second.mod) ctx->drv.ModuleUnload(p.second.mod);
    ctx->def_kernels.clear();
}

extern "C" {

kl_status kl_def_create(kl_def **out, const char *name, const char *source, const char *function)
{
    if (!out) return fail(KL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!name || !valid_ident(name)) return fail(KL_ERR_INVALID_ARG, "name must be a C identifier");
    if (!source || !*source || !function || !*function)
        return fail(KL_ERR_INVALID_ARG, "source and function are required");
    kl_def *d = new kl_def();
    d->name = name;
    d->source = source;
    d->function = function;
    *out = d;
    return KL_OK;
}

void kl_def_destroy(kl_def *d) { delete d; }

kl_status kl_def_param(kl_def *d, const char *name, int32_t n, const int64_t *values, int64_t dflt)
{
    if (!d || !name || !valid_ident(name)) return fail(KL_ERR_INVALID_ARG, "parameter name must be a C identifier");
    std::string nm = name;
    if (nm == "problem_x" || nm == "problem_y" || nm == "problem_z")
        return fail(KL_ERR_INVALID_ARG, "problem_x/y/z are reserved");
    for (auto &p : d->params)
        if (p.name == nm) return fail(KL_ERR_INVALID_ARG, "parameter '" + nm + "' declared twice");
    if (n < 1 || !values) return fail(KL_ERR_INVALID_ARG, "a parameter needs at least one value");
    std::vector<int64_t> v(values, values + n);
    std::set<int64_t> uniq(v.begin(), v.end());
    if (uniq.size() != v.size()) return fail(KL_ERR_INVALID_ARG, "parameter values must be distinct");
    if (!uniq.count(dflt)) return fail(KL_ERR_INVALID_ARG, "the default must be one of the values");
    d->params.push_back({nm, v, dflt});
    if (raw_size(*d) < 0) {
        d->params.pop_back();
        return fail(KL_ERR_INVALID_ARG, "configuration space too large");
    }
    return KL_OK;
}

kl_status kl_def_restrict(kl_def *d, const char *expr)
{
    if (!d || !expr) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    std::string err, text = expr;
    ExprP e = Parser(text).parse(&err);
    if (!e) return fail(KL_ERR_INVALID_ARG, "restriction: " + err);
    std::set<std::string> names;
    names_of(*e, &names);
    for (auto &n : names) {
        bool found = false;
        for (auto &p : d->params) found |= p.name == n;
        if (!found) return fail(KL_ERR_INVALID_ARG, "restriction uses '" + n + "', not a declared parameter");
    }
    d->restrictions.emplace_back(text, e);
    return KL_OK;
}

kl_status kl_def_geometry(kl_def *d, const char *const block[3], const char *const grid[3],
                          const char *shared_memory)
{
    if (!d) return fail(KL_ERR_INVALID_ARG, "NULL definition");
    const char *src[7] = {block ? block[0] : nullptr, block ? block[1] : nullptr,
                          block ? block[2] : nullptr, grid ? grid[0] : nullptr,
                          grid ? grid[1] : nullptr,   grid ? grid[2] : nullptr, shared_memory};
    ExprP parsed[7];
    for (int q = 0; q < 7; ++q) {
        if (!src[q] || !*src[q]) continue;
        std::string err, text = src[q];
        parsed[q] = Parser(text).parse(&err);
        if (!parsed[q]) return fail(KL_ERR_INVALID_ARG, std::string(kGeoNames[q]) + ": " + err);
    }
    for (int q = 0; q < 7; ++q) {
        d->geo[q] = parsed[q];
        d->geo_text[q] = src[q] && *src[q] ? src[q] : "";
    }
    return KL_OK;
}

kl_status kl_def_options(kl_def *d, const char *options)
{
    if (!d) return fail(KL_ERR_INVALID_ARG, "NULL definition");
    d->options = options ? options : "";
    return KL_OK;
}

kl_status kl_def_space_size(const kl_def *d, int64_t *raw, int64_t *valid)
{
    if (!d || !raw || !valid) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    *raw = raw_size(*d);
    *valid = -1;
    if (*raw <= 10000000) {
        int64_t n = 0;
        std::string err;
        for (int64_t i = 0; i < *raw; ++i)
            if (restrictions_hold(*d, values_at(*d, i), &err)) ++n;
        *valid = n;
    }
    return KL_OK;
}

kl_status kl_def_config_at(const kl_def *d, int64_t idx, char *buf, size_t n)
{
    if (!d || !buf || !n) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    if (idx < 0 || idx >= raw_size(*d)) return fail(KL_ERR_INVALID_ARG, "index outside the space");
    Values v = values_at(*d, idx);
    std::string s = config_text(*d, v), err;
    if (s.size() + 1 > n) return fail(KL_ERR_INVALID_ARG, "buffer too small");
    memcpy(buf, s.c_str(), s.size() + 1);
    if (!restrictions_hold(*d, v, &err)) return fail(KL_ERR_INVALID_ARG, err);
    return KL_OK;
}

kl_status kl_def_normalize(const kl_def *d, const char *config, char *buf, size_t n)
{
    if (!d || !config || !buf || !n) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    Values v;
    std::string err;
    if (!parse_config(*d, config, &v, &err) || !restrictions_hold(*d, v, &err))
        return fail(KL_ERR_INVALID_ARG, err);
    std::string s = config_text(*d, v);
    if (s.size() + 1 > n) return fail(KL_ERR_INVALID_ARG, "buffer too small");
    memcpy(buf, s.c_str(), s.size() + 1);
    return KL_OK;
}

kl_status kl_def_launch_geometry(const kl_def *d, const char *config, const int64_t problem[3],
                                 int64_t out[7])
{
    if (!d || !config || !problem || !out) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    Values v;
    std::string err;
    if (!parse_config(*d, config, &v, &err) || !restrictions_hold(*d, v, &err))
        return fail(KL_ERR_INVALID_ARG, err);
    if (!geometry(*d, v, problem, out, &err)) return fail(KL_ERR_INVALID_ARG, err);
    return KL_OK;
}

kl_status kl_def_compile_only(const kl_def *d, const char *config, char *log, size_t n)
{
    if (!d || !config) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    Values v;
    std::string err;
    if (!parse_config(*d, config, &v, &err) || !restrictions_hold(*d, v, &err))
        return fail(KL_ERR_INVALID_ARG, err);
    Compiled c;
    kl_status st = def_compile(*d, def_defines(*d, v), true, &c);
    if (log && n) {
        std::string s = st ? std::string(kl_last_error()) : c.log + "\nsymbol " + c.symbol;
        size_t m = std::min(n - 1, s.size());
        memcpy(log, s.data(), m);
        log[m] = '\0';
    }
    return st;
}

kl_status kl_def_launch_config(kl_ctx *ctx, kl_def *d, const char *config, const int64_t problem[3],
                               int32_t nargs, const kl_arg *args, void *stream)
{
    if (!ctx || !d || !config || !problem) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    kl_status st = check_args(nargs, args);
    if (st) return st;
    Values v;
    std::string err;
    if (!parse_config(*d, config, &v, &err)) return fail(KL_ERR_INVALID_ARG, err);
    return def_launch_values(ctx, d, v, problem, nargs, args, (cudaStream_t)stream);
}

kl_status kl_def_launch(kl_ctx *ctx, kl_def *d, const int64_t problem[3], int32_t nargs,
                        const kl_arg *args, void *stream)
{
    if (!ctx || !d || !problem) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    kl_status st = check_args(nargs, args);
    if (st) return st;
    char key[128];
    snprintf(key, sizeof key, "%p:%lld,%lld,%lld:", (void *)ctx, (long long)problem[0],
             (long long)problem[1], (long long)problem[2]);
    std::string skey = key + ctx->wisdom_dir;
    auto it = d->selection.find(skey);
    if (it == d->selection.end()) {
        // Sec. 4.5: the wisdom record of this device and problem size, else the
        // nearest size, else the same architecture, else any, else the default
        std::vector<WisdomRecord> recs;
        std::string err, text = "default";
        int rule = 5;
        if (wisdom_read(def_wisdom_path(ctx, *d), &recs, &err) && !recs.empty())
            rule = wisdom_select(recs, ctx->name, ctx->cc_major, ctx->cc_minor, 0,
                                 wisdom_extent(problem[0]), wisdom_extent(problem[1]),
                                 wisdom_extent(problem[2]), &text);
        Values v;
        int64_t geo[7];
        if (!parse_config(*d, text, &v, &err) || !restrictions_hold(*d, v, &err) ||
            !geometry(*d, v, problem, geo, &err)) {
            text = "default";
            rule = 5;
        }
        d->last_rule = rule;
        it = d->selection.emplace(skey, text).first;
    }
    Values v;
    std::string err;
    if (!parse_config(*d, it->second, &v, &err)) return fail(KL_ERR_INVALID_ARG, err);
    return def_launch_values(ctx, d, v, problem, nargs, args, (cudaStream_t)stream);
}

kl_status kl_def_selected(const kl_def *d, char *buf, size_t n, int32_t *rule)
{
    if (!d || !buf || !n || !rule) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    size_t m = std::min(n - 1, d->last_config.size());
    memcpy(buf, d->last_config.data(), m);
    buf[m] = '\0';
    *rule = d->last_rule;
    return KL_OK;
}

kl_status kl_def_capture(kl_ctx *ctx, const kl_def *d, const int64_t problem[3], int32_t nargs,
                         const kl_arg *args, const char *path, void *stream)
{
    if (!ctx || !d || !problem || !path) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    kl_status st = check_args(nargs, args);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "capture: synchronise");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(KL_ERR_IO, std::string("cannot write capture ") + path);
    // header: one field per line ("arg <index> <kind> <bytes> <dtype>"), then
    // the scalar values and input buffers in argument order
    fprintf(f, "KLDEFCAP1\nname %s\nfunction %s\nproblem %lld %lld %lld\nnargs %d\n", d->name.c_str(),
            d->function.c_str(), (long long)problem[0], (long long)problem[1], (long long)problem[2],
            nargs);
    fprintf(f, "device %s\ncc %d.%d\n", ctx->name.c_str(), ctx->cc_major, ctx->cc_minor);
    for (int q = 0; q < nargs; ++q)
        fprintf(f, "arg %d %d %lld %d\n", q, args[q].kind, (long long)args[q].bytes, args[q].dtype);
    fprintf(f, "END\n");
    bool ok = true;
    for (int q = 0; q < nargs && ok; ++q) {
        if (args[q].kind == 2) continue;       // outputs: only their size is recorded
        std::vector<char> b((size_t)args[q].bytes);
        if (args[q].kind == 0) {
            memcpy(b.data(), args[q].ptr, b.size());
        } else if (!b.empty()) {
            e = cudaMemcpy(b.data(), args[q].ptr, b.size(), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                fclose(f);
                return cuda_fail(e, "capture: copy");
            }
        }
        ok = fwrite(b.data(), 1, b.size(), f) == b.size();
    }
    ok = fclose(f) == 0 && ok;
    if (!ok) return fail(KL_ERR_IO, std::string("capture: write failed: ") + path);
    return KL_OK;
}

kl_status kl_def_tune(kl_ctx *ctx, kl_def *d, const char *capture_path, const char *opts,
                      const char *wisdom_path)
{
    if (!ctx || !d || !capture_path || !wisdom_path) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    DefOpts O;
    kl_status st = def_parse_opts(opts, &O);
    if (st) return st;
    auto t_start = std::chrono::steady_clock::now();
    auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    };
    DefCapture C;
    st = def_capture_read(capture_path, &C);
    if (st) return st;
    if (C.name != d->name || C.function != d->function)
        return fail(KL_ERR_INVALID_ARG, "capture is of " + C.name + " (" + C.function + "), not " + d->name);

    // device buffers of the replay (freed on every return)
    struct Bufs {
        std::vector<void *> p;
        ~Bufs() { for (void *x : p) cudaFree(x); }
    } B, Init;
    size_t na = C.args.size();
    B.p.assign(na, nullptr);
    Init.p.assign(na, nullptr);
    std::vector<kl_arg> args(na);
    for (size_t q = 0; q < na; ++q) {
        args[q] = C.args[q];
        if (C.args[q].kind == 0) {
            args[q].ptr = C.data[q].data();
            continue;
        }
        size_t nb = std::max<size_t>(1, (size_t)C.args[q].bytes);
        if (cudaMalloc(&B.p[q], nb) != cudaSuccess) return fail(KL_ERR_OOM, "tune: allocation failed");
        args[q].ptr = B.p[q];
        if (C.args[q].kind != 2 && C.args[q].bytes > 0 &&
            cudaMemcpy(B.p[q], C.data[q].data(), (size_t)C.args[q].bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(KL_ERR_CUDA, "tune: upload failed");
        if (C.args[q].kind == 3) {
            if (cudaMalloc(&Init.p[q], nb) != cudaSuccess) return fail(KL_ERR_OOM, "tune: allocation failed");
            cudaMemcpy(Init.p[q], B.p[q], (size_t)C.args[q].bytes, cudaMemcpyDeviceToDevice);
        }
    }
    // before every checked run: in/out buffers from their captured contents,
    // outputs filled with 0xff bytes (NaN for floats), so unwritten elements show
    auto reset = [&]() {
        for (size_t q = 0; q < na; ++q) {
            if (C.args[q].bytes <= 0) continue;
            if (C.args[q].kind == 3)
                cudaMemcpy(B.p[q], Init.p[q], (size_t)C.args[q].bytes, cudaMemcpyDeviceToDevice);
            if (C.args[q].kind == 2) cudaMemset(B.p[q], 0xff, (size_t)C.args[q].bytes);
        }
    };
    auto outputs = [&](std::vector<std::vector<char>> *out) -> bool {
        out->assign(na, {});
        for (size_t q = 0; q < na; ++q)
            if (C.args[q].kind >= 2 && C.args[q].bytes > 0) {
                (*out)[q].resize((size_t)C.args[q].bytes);
                if (cudaMemcpy((*out)[q].data(), B.p[q], (size_t)C.args[q].bytes, cudaMemcpyDeviceToHost) !=
                    cudaSuccess)
                    return false;
            }
        return true;
    };
    auto run_once = [&](const Values &v) -> kl_status {
        reset();
        kl_status s = def_launch_values(ctx, d, v, C.problem, (int32_t)na, args.data(), 0);
        if (s) return s;
        cudaError_t e = cudaDeviceSynchronize();
        return e == cudaSuccess ? KL_OK : cuda_fail(e, "tune: run");
    };
    auto time_values = [&](const Values &v, int warm, int reps, double *us) -> kl_status {
        std::vector<cudaEvent_t> ev(2 * reps);
        for (auto &x : ev) cudaEventCreate(&x);
        kl_status s = KL_OK;
        for (int q = 0; q < warm && !s; ++q) s = def_launch_values(ctx, d, v, C.problem, (int32_t)na, args.data(), 0);
        for (int q = 0; q < reps && !s; ++q) {
            cudaEventRecord(ev[2 * q], 0);
            s = def_launch_values(ctx, d, v, C.problem, (int32_t)na, args.data(), 0);
            cudaEventRecord(ev[2 * q + 1], 0);
        }
        cudaError_t e = cudaDeviceSynchronize();
        std::vector<float> ms;
        if (!s && e == cudaSuccess)
            for (int q = 0; q < reps; ++q) {
                float t = 0;
                cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]);
                ms.push_back(t);
            }
        for (auto &x : ev) cudaEventDestroy(x);
        if (s) return s;
        if (e != cudaSuccess) return cuda_fail(e, "tune: timing");
        std::sort(ms.begin(), ms.end());
        *us = 1e3 * ms[ms.size() / 2];
        return KL_OK;
    };

    // the default configuration's outputs are the reference
    Values def = default_values(*d);
    std::string err;
    int64_t geo[7];
    if (!restrictions_hold(*d, def, &err) || !geometry(*d, def, C.problem, geo, &err))
        return fail(KL_ERR_INVALID_ARG, "the default configuration does not apply: " + err);
    st = run_once(def);
    if (st) return st;
    std::vector<std::vector<char>> ref;
    if (!outputs(&ref)) return fail(KL_ERR_CUDA, "tune: read back");
    double def_us = INFINITY;
    st = time_values(def, O.warm, O.reps, &def_us);
    if (st) return st;

    // candidates
    std::mt19937_64 rng(O.seed);
    int64_t raw = raw_size(*d);
    std::set<std::string> queued;
    auto applies = [&](const Values &v) {
        std::string e2;
        int64_t g2[7];
        return restrictions_hold(*d, v, &e2) && geometry(*d, v, C.problem, g2, &e2);
    };
    auto draw_random = [&](Values *v) {
        for (int tries = 0; tries < 100000; ++tries) {
            *v = values_at(*d, (int64_t)(rng() % (uint64_t)raw));
            if (applies(*v) && !queued.count(config_text(*d, *v))) return true;
        }
        return false;
    };
    int64_t ex_next = 0;
    auto draw_exhaustive = [&](Values *v) {
        while (ex_next < raw) {
            *v = values_at(*d, ex_next++);
            if (applies(*v) && !queued.count(config_text(*d, *v))) return true;
        }
        return false;
    };
    // features for the surrogate: each parameter's value index scaled to [0, 1]
    auto features = [&](const Values &v, double *f) {
        for (size_t q = 0; q < d->params.size(); ++q) {
            auto &vals = d->params[q].values;
            size_t i = (size_t)(std::find(vals.begin(), vals.end(), v[q]) - vals.begin());
            f[q] = vals.size() > 1 ? (double)i / (vals.size() - 1) : 0.0;
        }
    };
    struct Eval {
        Values v;
        double us = INFINITY, err = INFINITY;
        bool ok = false;
        std::string note;
    };
    std::vector<Eval> evals;
    const int bo_initial = std::max(4, std::min(16, O.max_evals / 6));
    auto propose_bayes = [&](const std::vector<Values> &pending, Values *out) {
        size_t dim = std::max<size_t>(1, d->params.size());
        std::vector<double> X, y, P, Cc, f(dim, 0.0);
        for (auto &e : evals)
            if (e.ok) {
                features(e.v, f.data());
                X.insert(X.end(), f.begin(), f.end());
                y.push_back(std::log(e.us));
            }
        if (y.size() < 2) return false;
        for (auto &v : pending) {
            features(v, f.data());
            P.insert(P.end(), f.begin(), f.end());
        }
        std::vector<Values> pool;
        std::set<std::string> in_pool;
        if (raw <= 4096) {
            for (int64_t i = 0; i < raw; ++i) {
                Values v = values_at(*d, i);
                std::string s = config_text(*d, v);
                if (applies(v) && !queued.count(s) && in_pool.insert(s).second) pool.push_back(v);
            }
        } else {
            for (int q = 0; q < 1024; ++q) {
                Values v;
                if (!draw_random(&v)) break;
                if (in_pool.insert(config_text(*d, v)).second) pool.push_back(v);
            }
        }
        if (pool.empty()) return false;
        for (auto &v : pool) {
            features(v, f.data());
            Cc.insert(Cc.end(), f.begin(), f.end());
        }
        std::vector<double> ei;
        std::string e2;
        int pick = bo_suggest((int)y.size(), (int)dim, X.data(), y.data(), (int)pending.size(), P.data(),
                              (int)pool.size(), Cc.data(), 0.01, 0.0, 0.0, nullptr, &ei, &e2);
        if (pick < 0) return false;
        *out = pool[(size_t)pick];
        return true;
    };
    int nthreads = O.threads > 0 ? O.threads
                   : std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
    FILE *logf = O.log.empty() ? nullptr : fopen(O.log.c_str(), "a");
    while (elapsed() < O.budget_s && (int)evals.size() < O.max_evals) {
        // a batch of candidates, compiled in parallel on host threads
        std::vector<Values> batch;
        int want = std::min(nthreads, O.max_evals - (int)evals.size());
        while ((int)batch.size() < want) {
            Values v;
            bool got = false;
            if (O.strategy == "exhaustive") got = draw_exhaustive(&v);
            else if (O.strategy == "bayes" && (int)(evals.size() + batch.size()) >= bo_initial)
                got = propose_bayes(batch, &v) || draw_random(&v);
            else got = draw_random(&v);
            if (!got) break;
            queued.insert(config_text(*d, v));
            batch.push_back(v);
        }
        if (batch.empty()) break;
        std::vector<std::future<std::pair<kl_status, Compiled>>> futs;
        for (auto &v : batch) {
            std::string defines = def_defines(*d, v);
            std::string ident = cache_identity(def_hash(*d), defines);
            bool have = ctx->def_kernels.count(ident) > 0;
            futs.push_back(std::async(std::launch::async, [d, defines, have]() {
                Compiled c;
                kl_status s = have ? KL_OK : def_compile(*d, defines, false, &c);
                return std::make_pair(s, std::move(c));
            }));
        }
        for (size_t b = 0; b < batch.size(); ++b) {
            auto res = futs[b].get();
            Eval e;
            e.v = batch[b];
            std::string ident = cache_identity(def_hash(*d), def_defines(*d, e.v));
            DefKernel *k = nullptr;
            kl_status s = res.first;
            if (s == KL_OK && !ctx->def_kernels.count(ident)) s = def_load(ctx, ident, res.second, &k);
            if (s == KL_OK) s = run_once(e.v);
            std::vector<std::vector<char>> got;
            if (s == KL_OK && !outputs(&got)) s = fail(KL_ERR_CUDA, "tune: read back");
            if (s == KL_OK) {
                // worst output relative to its tolerance (verify_tol, else by dtype)
                e.err = 0;
                e.ok = true;
                for (size_t q = 0; q < na; ++q)
                    if (C.args[q].kind >= 2) {
                        double x = compare(C.args[q].dtype, got[q], ref[q]);
                        double tol = O.verify_tol >= 0 ? O.verify_tol : default_tol(C.args[q].dtype);
                        e.err = std::max(e.err, x);
                        e.ok = e.ok && x <= tol;
                    }
                if (!e.ok) e.note = "verification failed";
                else s = time_values(e.v, O.warm, O.reps, &e.us);
            }
            if (s != KL_OK) {
                e.ok = false;
                e.note = kl_last_error();
                if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
                    if (logf) fclose(logf);
                    return fail(KL_ERR_CUDA, "tune: device error, stopping: " + e.note);
                }
            }
            if (logf) {
                std::string note;
                for (char ch : e.note) note += ch == '"' ? '\'' : ch == '\n' ? ' ' : ch;
                fprintf(logf, "{\"config\":\"%s\",\"time_us\":%.4f,\"err\":%.3e,\"ok\":%s,\"t_s\":%.3f,\"note\":\"%s\"}\n",
                        config_text(*d, e.v).c_str(), e.ok ? e.us : -1.0, std::isfinite(e.err) ? e.err : -1.0,
                        e.ok ? "true" : "false", elapsed(), note.c_str());
                fflush(logf);
            }
            evals.push_back(e);
        }
    }
    if (logf) fclose(logf);

    // re-time the three fastest and keep the best (the default if nothing beats it)
    std::vector<Eval> ok;
    for (auto &e : evals)
        if (e.ok) ok.push_back(e);
    std::sort(ok.begin(), ok.end(), [](const Eval &a, const Eval &b) { return a.us < b.us; });
    if (ok.size() > 3) ok.resize(3);
    Values best = def;
    double best_us = def_us;
    st = time_values(def, O.warm, 3 * O.reps, &best_us);
    if (st) return st;
    def_us = best_us;
    for (auto &e : ok) {
        double t;
        st = time_values(e.v, O.warm, 3 * O.reps, &t);
        if (st) return st;
        if (t < best_us) {
            best_us = t;
            best = e.v;
        }
    }
    WisdomRecord rec;
    rec.device = ctx->name;
    rec.cc_major = ctx->cc_major;
    rec.cc_minor = ctx->cc_minor;
    rec.zbc = 0;
    rec.nx = wisdom_extent(C.problem[0]);
    rec.ny = wisdom_extent(C.problem[1]);
    rec.nz = wisdom_extent(C.problem[2]);
    rec.config = config_text(*d, best);
    rec.time_us = best_us;
    char buf[64];
    time_t now = time(nullptr);
    struct tm tmv;
    gmtime_r(&now, &tmv);
    strftime(buf, sizeof buf, "%Y-%m-%dT%H:%M:%SZ", &tmv);
    rec.extra["date"] = buf;
    rec.extra["kernel"] = d->name;
    rec.extra["strategy"] = O.strategy;
    rec.extra["evals"] = std::to_string(evals.size());
    snprintf(buf, sizeof buf, "%.1f", elapsed());
    rec.extra["tune_s"] = buf;
    snprintf(buf, sizeof buf, "%.3f", def_us);
    rec.extra["default_us"] = buf;
    snprintf(buf, sizeof buf, "%.3f", best_us > 0 ? def_us / best_us : 1.0);
    rec.extra["speedup"] = buf;
    rec.extra["sms"] = std::to_string(ctx->nsm);
    if (!wisdom_append(wisdom_path, rec, &err)) return fail(KL_ERR_IO, err);
    d->selection.clear();      // the next kl_def_launch reads the wisdom again
    return KL_OK;
}

}  // extern "C"
