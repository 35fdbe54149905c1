// kl_tune.cpp -- capture (Sec. 4.2), tuning (Sec. 4.3) with wisdom output
// (Sec. 4.4), and batched launches over many grids.
#include <nvrtc.h>
#include <unistd.h>

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <fstream>
#include <future>
#include <random>
#include <set>
#include <sstream>
#include <thread>

#include "kl_internal.h"

namespace kl {

// ================================================================ helpers

static std::string now_iso()
{
    time_t t = time(nullptr);
    struct tm g;
    gmtime_r(&t, &g);
    char b[32];
    strftime(b, sizeof b, "%Y-%m-%dT%H:%M:%SZ", &g);
    return b;
}

static std::string host_name()
{
    char b[256] = {0};
    if (gethostname(b, sizeof b - 1) != 0) return "unknown";
    return b;
}

static const char *dtype_tag(int d)
{
    return d == KL_F64 ? "f64" : d == KL_F32 ? "f32" : d == KL_BF16 ? "bf16" : "f16";
}

// ================================================================ capture
//
// File layout: a text header of key=value lines ending with "END\n", then the
// raw device buffers (each `extent` elements of the storage type) in the order
// the header's blobs= line lists.  The header carries the kernel definition
// (op), the problem (grid, layout, scalars, vertical grid) and provenance.

struct Capture {
    kl_op op;
    kl_grid grid;
    std::vector<double> zh;
    std::string device;
    int cc_major = 0, cc_minor = 0;
    std::vector<std::string> names;
    size_t blob_bytes = 0;          // u, v, w, nu
    size_t out_bytes = 0;           // ut, vt, wt (accumulate)
    std::vector<std::vector<char>> blobs;
};

static std::vector<std::string> capture_blob_names(const kl_op &op)
{
    std::vector<std::string> n = {"u", "v", "w"};
    if (op.diff == 2) n.push_back("nu");
    if (op.accumulate) {
        n.push_back("ut");
        n.push_back("vt");
        n.push_back("wt");
    }
    return n;
}

kl_status capture_write(kl_ctx *ctx, const kl_op &op, const kl_grid &g, const kl_fields &f,
                        const std::string &path, cudaStream_t s)
{
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "capture: stream sync");
    std::vector<std::string> names = capture_blob_names(op);
    std::map<std::string, const void *> ptr = {{"u", f.u}, {"v", f.v}, {"w", f.w}, {"nu", f.nu},
                                                {"ut", f.ut}, {"vt", f.vt}, {"wt", f.wt}};
    size_t bytes = (size_t)g.extent * esize_of(op.dtype);
    size_t obytes = (size_t)g.extent * esize_of(out_dtype(op));
    FILE *out = fopen(path.c_str(), "wb");
    if (!out) return fail(KL_ERR_IO, "capture: cannot open " + path);
    fprintf(out, "KLCAPTURE 1\n");
    fprintf(out, "kernel=tendency adv=%d diff=%d dtype=%d accumulate=%d out_f32=%d\n", op.adv,
            op.diff, op.dtype, op.accumulate, op.out_f32);
    fprintf(out, "nx=%d ny=%d nz=%d g=%d sj=%lld sk=%lld origin=%lld extent=%lld zbc=%d\n", g.nx,
            g.ny, g.nz, g.g, (long long)g.sj, (long long)g.sk, (long long)g.origin,
            (long long)g.extent, g.zbc);
    fprintf(out, "dx=%.17g dy=%.17g dz=%.17g nu=%.17g\n", g.dx, g.dy, g.dz, g.nu);
    fprintf(out, "zh=%d", g.zh ? g.nz + 1 : 0);
    if (g.zh)
        for (int k = 0; k <= g.nz; ++k) fprintf(out, " %.17g", g.zh[k]);
    fprintf(out, "\n");
    fprintf(out, "device=\"%s\" cc=%d.%d date=%s host=%s\n", ctx->name.c_str(), ctx->cc_major,
            ctx->cc_minor, now_iso().c_str(), host_name().c_str());
    std::string list;
    for (auto &n : names) list += (list.empty() ? "" : ",") + n;
    fprintf(out, "blobs=%s bytes=%zu obytes=%zu\nEND\n", list.c_str(), bytes, obytes);
    std::vector<char> host(std::max(bytes, obytes));
    for (auto &n : names) {
        const size_t nb = (n == "ut" || n == "vt" || n == "wt") ? obytes : bytes;
        e = cudaMemcpy(host.data(), ptr[n], nb, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            fclose(out);
            return cuda_fail(e, "capture: device to host copy");
        }
        if (fwrite(host.data(), 1, nb, out) != nb) {
            fclose(out);
            return fail(KL_ERR_IO, "capture: short write to " + path);
        }
    }
    if (fclose(out) != 0) return fail(KL_ERR_IO, "capture: close failed for " + path);
    return KL_OK;
}

static bool kv_line(const std::string &line, std::map<std::string, std::string> *kv)
{
    std::stringstream ss(line);
    std::string tok;
    bool any = false;
    // values are single tokens except device="..." which may hold spaces
    size_t p = 0;
    while (p < line.size()) {
        while (p < line.size() && line[p] == ' ') ++p;
        size_t eq = line.find('=', p);
        if (eq == std::string::npos) break;
        std::string k = line.substr(p, eq - p);
        p = eq + 1;
        std::string v;
        if (p < line.size() && line[p] == '"') {
            size_t q = line.find('"', p + 1);
            if (q == std::string::npos) return false;
            v = line.substr(p + 1, q - p - 1);
            p = q + 1;
        } else {
            size_t q = line.find(' ', p);
            if (q == std::string::npos) q = line.size();
            v = line.substr(p, q - p);
            p = q;
        }
        (*kv)[k] = v;
        any = true;
    }
    return any;
}

kl_status capture_read(const std::string &path, Capture *c)
{
    FILE *in = fopen(path.c_str(), "rb");
    if (!in) return fail(KL_ERR_IO, "capture: cannot open " + path);
    std::map<std::string, std::string> kv;
    std::vector<double> zh;
    char line[1 << 16];
    bool magic = false, end = false;
    while (fgets(line, sizeof line, in)) {
        std::string l(line);
        while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
        if (!magic) {
            if (l != "KLCAPTURE 1") break;
            magic = true;
            continue;
        }
        if (l == "END") {
            end = true;
            break;
        }
        if (l.rfind("zh=", 0) == 0) {
            std::stringstream ss(l.substr(3));
            int n = 0;
            ss >> n;
            for (int q = 0; q < n; ++q) {
                double x;
                if (!(ss >> x)) break;
                zh.push_back(x);
            }
            if ((int)zh.size() != n) {
                fclose(in);
                return fail(KL_ERR_WISDOM_PARSE, "capture: bad zh line");
            }
            continue;
        }
        kv_line(l, &kv);
    }
    if (!magic || !end) {
        fclose(in);
        return fail(KL_ERR_WISDOM_PARSE, "capture: not a capture file: " + path);
    }
    auto geti = [&](const char *k, long long *v) {
        auto it = kv.find(k);
        if (it == kv.end()) return false;
        char *e = nullptr;
        *v = strtoll(it->second.c_str(), &e, 10);
        return e && *e == 0;
    };
    auto getd = [&](const char *k, double *v) {
        auto it = kv.find(k);
        if (it == kv.end()) return false;
        char *e = nullptr;
        *v = strtod(it->second.c_str(), &e);
        return e && *e == 0;
    };
    long long adv, diff, dtype, acc, nx, ny, nz, g, sj, sk, origin, extent, zbc;
    double dx, dy, dz, nu;
    long long bytes;
    if (!geti("adv", &adv) || !geti("diff", &diff) || !geti("dtype", &dtype) ||
        !geti("accumulate", &acc) || !geti("nx", &nx) || !geti("ny", &ny) || !geti("nz", &nz) ||
        !geti("g", &g) || !geti("sj", &sj) || !geti("sk", &sk) || !geti("origin", &origin) ||
        !geti("extent", &extent) || !geti("zbc", &zbc) || !getd("dx", &dx) || !getd("dy", &dy) ||
        !getd("dz", &dz) || !getd("nu", &nu) || !geti("bytes", &bytes)) {
        fclose(in);
        return fail(KL_ERR_WISDOM_PARSE, "capture: header lacks a field: " + path);
    }
    long long of32 = 0, obytes = 0;
    if (!geti("out_f32", &of32)) of32 = 0;          // captures written before the field
    c->op = kl_op{(int)adv, (int)diff, (int)dtype, (int)acc, (int)of32};
    if (!geti("obytes", &obytes)) obytes = (long long)extent * esize_of(out_dtype(c->op));
    c->zh = zh;
    kl_grid &G = c->grid;
    memset(&G, 0, sizeof G);
    G.nx = (int)nx; G.ny = (int)ny; G.nz = (int)nz; G.g = (int)g;
    G.sj = sj; G.sk = sk; G.origin = origin; G.extent = extent; G.zbc = (int)zbc;
    G.dx = dx; G.dy = dy; G.dz = dz; G.nu = nu;
    G.zh = nullptr;   // set by the user of the capture (points into c->zh)
    if (!zh.empty() && (int)zh.size() != nz + 1) {
        fclose(in);
        return fail(KL_ERR_WISDOM_PARSE, "capture: zh has the wrong length");
    }
    c->device = kv["device"];
    sscanf(kv["cc"].c_str(), "%d.%d", &c->cc_major, &c->cc_minor);
    std::stringstream ss(kv["blobs"]);
    std::string n;
    while (std::getline(ss, n, ',')) c->names.push_back(n);
    if (c->names != capture_blob_names(c->op) ||
        (size_t)bytes != (size_t)extent * esize_of((int)dtype) ||
        (size_t)obytes != (size_t)extent * esize_of(out_dtype(c->op))) {
        fclose(in);
        return fail(KL_ERR_WISDOM_PARSE, "capture: blob list or size does not match the op");
    }
    c->blob_bytes = (size_t)bytes;
    c->out_bytes = (size_t)obytes;
    for (size_t q = 0; q < c->names.size(); ++q) {
        const std::string &bn = c->names[q];
        std::vector<char> b(bn == "ut" || bn == "vt" || bn == "wt" ? c->out_bytes : c->blob_bytes);
        if (fread(b.data(), 1, b.size(), in) != b.size()) {
            fclose(in);
            return fail(KL_ERR_WISDOM_PARSE, "capture: truncated data in " + path);
        }
        c->blobs.push_back(std::move(b));
    }
    fclose(in);
    return KL_OK;
}

// ================================================================= tuner

struct TuneOpts {
    std::string strategy = "random";
    double budget_s = 60;
    int max_evals = 200;
    unsigned seed = 1;
    std::string family = "all";
    double verify_tol = -1;
    std::string log;
    int reps = 7;
    int warm = 2;
    int topk = 3;
    int threads = 0;
};

static kl_status parse_opts(const char *text, TuneOpts *o)
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
        else if (k == "family") o->family = v;
        else if (k == "verify_tol") o->verify_tol = atof(v.c_str());
        else if (k == "log") o->log = v;
        else if (k == "reps") o->reps = std::max(1, atoi(v.c_str()));
        else if (k == "warm") o->warm = std::max(0, atoi(v.c_str()));
        else if (k == "topk") o->topk = std::max(1, atoi(v.c_str()));
        else if (k == "threads") o->threads = atoi(v.c_str());
        else return fail(KL_ERR_INVALID_ARG, "unknown tune option '" + k + "'");
    }
    if (o->strategy != "random" && o->strategy != "exhaustive" && o->strategy != "local" &&
        o->strategy != "bayes")
        return fail(KL_ERR_INVALID_ARG, "strategy must be random, exhaustive, local or bayes");
    if (o->family != "all" && o->family != "direct" && o->family != "zmarch" && o->family != "zpack")
        return fail(KL_ERR_INVALID_ARG, "family must be all, direct, zmarch or zpack");
    return KL_OK;
}

// device buffers of one replay
struct Replay {
    std::vector<void *> in;        // u, v, w, nu (nu may be null)
    void *out[3] = {nullptr, nullptr, nullptr};
    void *ref[3] = {nullptr, nullptr, nullptr};
    void *init[3] = {nullptr, nullptr, nullptr};   // accumulate: pristine outputs
    unsigned long long *cmp = nullptr;
    size_t bytes = 0, obytes = 0;
    ~Replay()
    {
        for (void *p : in) cudaFree(p);
        for (int q = 0; q < 3; ++q) {
            cudaFree(out[q]);
            cudaFree(ref[q]);
            cudaFree(init[q]);
        }
        cudaFree(cmp);
    }
};

struct Eval {
    std::string config;
    double time_us = INFINITY;
    double err = INFINITY;
    bool ok = false;
    std::string note;
};

static std::string json_escape(const std::string &s)
{
    std::string o;
    for (char ch : s) {
        if (ch == '"' || ch == '\\') o += '\\';
        if (ch == '\n') { o += "\\n"; continue; }
        o += ch;
    }
    return o;
}

static void log_eval(const std::string &path, const Eval &e, double t)
{
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "{\"config\":\"%s\",\"time_us\":%.4f,\"err\":%.3e,\"ok\":%s,\"t_s\":%.3f,\"note\":\"%s\"}\n",
            e.config.c_str(), std::isfinite(e.time_us) ? e.time_us : -1.0,
            std::isfinite(e.err) ? e.err : -1.0, e.ok ? "true" : "false", t,
            json_escape(e.note).c_str());
    fclose(f);
}

// previously evaluated configurations of a session (resume after a kill)
static void read_log(const std::string &path, std::map<std::string, Eval> *done)
{
    if (path.empty()) return;
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
        auto grab = [&](const char *key) -> std::string {
            std::string k = std::string("\"") + key + "\":";
            size_t p = line.find(k);
            if (p == std::string::npos) return "";
            p += k.size();
            if (line[p] == '"') {
                size_t q = line.find('"', p + 1);
                return line.substr(p + 1, q - p - 1);
            }
            size_t q = line.find_first_of(",}", p);
            return line.substr(p, q - p);
        };
        Eval e;
        e.config = grab("config");
        if (e.config.empty()) continue;
        double t = atof(grab("time_us").c_str());
        e.time_us = t > 0 ? t : INFINITY;
        double er = atof(grab("err").c_str());
        e.err = er >= 0 ? er : INFINITY;
        e.ok = grab("ok") == "true";
        e.note = "resumed";
        (*done)[e.config] = e;
    }
}

// time one configuration: median of `reps` launches after `warm` launches
static kl_status time_config(kl_ctx *ctx, const kl_op &op, const Config &cfg, const kl_grid &g,
                             Replay &R, int warm, int reps, double *median_us)
{
    kl_fields f{R.in[0], R.in[1], R.in[2], R.in.size() > 3 ? R.in[3] : nullptr, R.out[0],
                R.out[1], R.out[2]};
    cudaStream_t s = 0;
    std::vector<cudaEvent_t> ev(2 * reps);
    for (auto &e : ev) cudaEventCreate(&e);
    kl_status st = KL_OK;
    for (int q = 0; q < warm && !st; ++q) st = launch_config(ctx, op, cfg, g, f, s);
    for (int q = 0; q < reps && !st; ++q) {
        cudaEventRecord(ev[2 * q], s);
        st = launch_config(ctx, op, cfg, g, f, s);
        cudaEventRecord(ev[2 * q + 1], s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    std::vector<float> ms;
    if (!st && e == cudaSuccess)
        for (int q = 0; q < reps; ++q) {
            float t = 0;
            cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]);
            ms.push_back(t);
        }
    for (auto &x : ev) cudaEventDestroy(x);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "tune: launch");
    std::sort(ms.begin(), ms.end());
    *median_us = 1e3 * ms[ms.size() / 2];
    return KL_OK;
}

// relative error of the candidate outputs against the reference outputs
static kl_status verify(kl_ctx *ctx, const kl_op &op, const kl_grid &g, Replay &R, double *err)
{
    double worst = 0;
    for (int q = 0; q < 3; ++q) {
        cudaError_t e = compare_launch(out_dtype(op), g, R.out[q], R.ref[q], R.cmp, ctx->nsm, 0);
        unsigned long long h[2];
        if (e == cudaSuccess) e = cudaMemcpy(h, R.cmp, sizeof h, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "tune: verify");
        double d, m;
        memcpy(&d, &h[0], 8);
        memcpy(&m, &h[1], 8);
        double r = m > 0 ? d / m : d;
        worst = std::max(worst, r);
    }
    *err = worst;
    return KL_OK;
}

static kl_status reset_outputs(const kl_op &op, Replay &R)
{
    if (!op.accumulate) return KL_OK;
    for (int q = 0; q < 3; ++q) {
        cudaError_t e = cudaMemcpy(R.out[q], R.init[q], R.obytes, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "tune: reset outputs");
    }
    return KL_OK;
}

// candidate generation ---------------------------------------------------

static bool valid_for(const kl_op &op, const kl_grid &g, int family, int64_t idx, Config *c)
{
    if (!space_config(family, idx, c)) return false;
    std::string err;
    return config_check(op, *c, &err) && config_fits(op, *c, g, nullptr, &err);
}

static std::vector<int> radices(int family)
{
    if (family == 0) return {5, 5, 5, 3, 3, 3, 2, 2, 2, 2, 2, 2, 6, 6};
    if (family == 2) return {10, 7, 7, 6, 4, 3, 2, 3};
    return {3, 5, 3, 3, 7, 4, 4};
}

static std::vector<int64_t> neighbours(int family, int64_t idx)
{
    std::vector<int> r = radices(family);
    std::vector<int> d(r.size());
    int64_t x = idx;
    for (size_t q = 0; q < r.size(); ++q) {
        d[q] = (int)(x % r[q]);
        x /= r[q];
    }
    std::vector<int64_t> out;
    for (size_t q = 0; q < r.size(); ++q)
        for (int step : {-1, 1}) {
            int v = d[q] + step;
            if (v < 0 || v >= r[q]) continue;
            std::vector<int> e = d;
            e[q] = v;
            int64_t y = 0;
            for (size_t p = r.size(); p-- > 0;) y = y * r[p] + e[p];
            out.push_back(y);
        }
    return out;
}

// the digits of a configuration in its family's raw space (inverse of
// space_config); false if a value is not one of the space's
static bool config_digits(const Config &c, std::vector<int> *digits)
{
    std::vector<std::vector<int>> vals;
    if (c.family == 0)
        vals = {{16, 32, 64, 128, 256}, {1, 2, 4, 8, 16}, {1, 2, 4, 8, 16}, {1, 2, 4}, {1, 2, 4},
                {1, 2, 4}, {0, 1}, {0, 1}, {0, 1}, {0, 1}, {0, 1}, {0, 1}, {0, 1, 2, 3, 4, 5},
                {1, 2, 3, 4, 5, 6}};
    else if (c.family == 2)
        vals = {{1, 2, 3, 4, 6, 7, 8, 9, 12, 16}, {1, 2, 3, 4, 5, 6, 8}, {4, 8, 16, 32, 64, 128, 256},
                {6, 7, 8, 9, 10, 12}, {1, 2, 3, 4}, {0, 1, 2}, {0, 1}, {0, 1, 2}};
    else
        vals = {{32, 64, 128}, {1, 2, 4, 8, 16}, {1, 2, 4}, {1, 2, 4}, {4, 8, 16, 32, 64, 128, 256},
                {8, 9, 10, 12}, {1, 2, 3, 4}};
    std::vector<int> cur = c.family == 0
        ? std::vector<int>{c.bx, c.by, c.bz, c.tx, c.ty, c.tz, c.ux, c.uy, c.uz, c.cx, c.cy, c.cz, c.perm, c.minb}
        : c.family == 2 ? std::vector<int>{c.mby, c.mpy, c.kc, c.ns, c.mminb, c.yx, c.cs, c.pe}
                        : std::vector<int>{c.mbx, c.mby, c.mpx, c.mpy, c.kc, c.ns, c.mminb};
    digits->resize(vals.size());
    for (size_t p = 0; p < vals.size(); ++p) {
        auto it = std::find(vals[p].begin(), vals[p].end(), cur[p]);
        if (it == vals[p].end()) return false;
        (*digits)[p] = (int)(it - vals[p].begin());
    }
    return true;
}

// Surrogate features of a configuration: a one-hot of the family (3 values),
// then one block per family (14 direct, 7 zmarch, 8 zpack digits), the
// configuration's own block holding each digit scaled to [0, 1] and the others
// zero.  The value lists of the space are ordered (powers of two, counts), so
// neighbouring digits are neighbouring settings.
static const int kFeatDims = 3 + 14 + 7 + 8;

static bool config_features(const Config &c, double *f)
{
    std::vector<int> dg;
    if (!config_digits(c, &dg)) return false;
    std::vector<int> r = radices(c.family);
    std::fill(f, f + kFeatDims, 0.0);
    f[c.family] = 1.0;
    int off = 3 + (c.family == 0 ? 0 : c.family == 1 ? 14 : 21);
    for (size_t q = 0; q < dg.size(); ++q) f[off + q] = r[q] > 1 ? (double)dg[q] / (r[q] - 1) : 0.0;
    return true;
}

}  // namespace kl

using namespace kl;

extern "C" {

kl_status kl_capture(kl_ctx *ctx, const kl_op *op, const kl_grid *grid, const kl_fields *fields,
                     const char *path, void *stream)
{
    if (!ctx || !op || !grid || !fields || !path) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    kl_status st = check_grid(grid, halo_of(*op), nullptr);
    if (st) return st;
    if (!fields->u || !fields->v || !fields->w || (op->diff == 2 && !fields->nu) ||
        (op->accumulate && (!fields->ut || !fields->vt || !fields->wt)))
        return fail(KL_ERR_INVALID_ARG, "capture: a needed field pointer is NULL");
    return capture_write(ctx, *op, *grid, *fields, path, (cudaStream_t)stream);
}

// called by kl_launch when $KERNEL_LAUNCHER_CAPTURE lists "tendency": one
// capture per problem per process, into $KL_CAPTURE_DIR
kl_status kl_capture_if_requested(kl_ctx *ctx, const kl_op *op, const kl_grid *grid,
                                  const kl_fields *fields, void *stream)
{
    char name[256];
    snprintf(name, sizeof name, "tendency_adv%d_diff%d_%s%s_%dx%dx%d_zbc%d.klcap", op->adv,
             op->diff, dtype_tag(op->dtype), op->accumulate ? "_acc" : "", grid->nx, grid->ny,
             grid->nz, grid->zbc);
    std::string key = std::string("capture:") + name;
    if (ctx->selection.count(key)) return KL_OK;
    const char *dir = getenv("KL_CAPTURE_DIR");
    std::string path = std::string(dir && *dir ? dir : ".") + "/" + name;
    kl_status st = capture_write(ctx, *op, *grid, *fields, path, (cudaStream_t)stream);
    if (st) return st;
    ctx->selection[key] = path;
    return KL_OK;
}

kl_status kl_tune(kl_ctx *ctx, const char *capture_path, const char *opts, const char *wisdom_path)
{
    if (!ctx || !capture_path || !wisdom_path) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    TuneOpts O;
    kl_status st = parse_opts(opts, &O);
    if (st) return st;
    auto t_start = std::chrono::steady_clock::now();
    auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    };
    Capture C;
    st = capture_read(capture_path, &C);
    if (st) return st;
    kl_op op = C.op;
    kl_grid g = C.grid;
    if (!C.zh.empty()) g.zh = C.zh.data();
    st = check_grid(&g, halo_of(op), nullptr);
    if (st) return st;

    // device buffers
    Replay R;
    R.bytes = C.blob_bytes;
    R.obytes = C.out_bytes;
    auto alloc = [&](void **p) { return cudaMalloc(p, R.bytes); };
    auto alloc_out = [&](void **p) { return cudaMalloc(p, R.obytes); };
    size_t nin = op.diff == 2 ? 4 : 3;
    for (size_t q = 0; q < nin; ++q) {
        void *p = nullptr;
        if (alloc(&p) != cudaSuccess) return fail(KL_ERR_OOM, "tune: device allocation failed");
        R.in.push_back(p);
        if (cudaMemcpy(p, C.blobs[q].data(), R.bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(KL_ERR_CUDA, "tune: upload failed");
    }
    for (int q = 0; q < 3; ++q) {
        if (alloc_out(&R.out[q]) != cudaSuccess || alloc_out(&R.ref[q]) != cudaSuccess)
            return fail(KL_ERR_OOM, "tune: device allocation failed");
        cudaMemset(R.out[q], 0, R.obytes);
        cudaMemset(R.ref[q], 0, R.obytes);
        if (op.accumulate) {
            if (alloc_out(&R.init[q]) != cudaSuccess) return fail(KL_ERR_OOM, "tune: allocation failed");
            cudaMemcpy(R.init[q], C.blobs[nin + q].data(), R.obytes, cudaMemcpyHostToDevice);
            cudaMemcpy(R.ref[q], R.init[q], R.obytes, cudaMemcpyDeviceToDevice);
        }
    }
    if (cudaMalloc(&R.cmp, 2 * sizeof(unsigned long long)) != cudaSuccess)
        return fail(KL_ERR_OOM, "tune: allocation failed");

    // reference output: the default configuration, launched once
    Config def;
    {
        kl_fields f{R.in[0], R.in[1], R.in[2], nin > 3 ? R.in[3] : nullptr, R.ref[0], R.ref[1], R.ref[2]};
        st = launch_config(ctx, op, def, g, f, 0);
        if (st) return st;
        if (cudaDeviceSynchronize() != cudaSuccess) return fail(KL_ERR_CUDA, "tune: reference run failed");
    }
    double tol = O.verify_tol > 0 ? O.verify_tol
                 : op.dtype == KL_F64 ? 1e-10 : out_dtype(op) == KL_F32 ? 1e-4 : 2e-2;

    // candidates
    std::mt19937_64 rng(O.seed);
    std::vector<int> fams;
    if (O.family == "all" || O.family == "direct") fams.push_back(0);
    if (O.family == "all" || O.family == "zmarch") fams.push_back(1);
    if (O.family == "all" || O.family == "zpack") fams.push_back(2);
    if (fams.empty()) return fail(KL_ERR_INVALID_ARG, "no configuration family applies to this op");
    std::map<std::string, Eval> done;
    read_log(O.log, &done);
    std::set<std::string> queued;
    for (auto &p : done) queued.insert(p.first);
    auto draw_random = [&](Config *c) {
        for (int tries = 0; tries < 100000; ++tries) {
            int fam = fams[rng() % fams.size()];
            int64_t idx = (int64_t)(rng() % (uint64_t)space_size(fam));
            if (valid_for(op, g, fam, idx, c)) {
                std::string s = config_string(*c);
                if (!queued.count(s)) return true;
            }
        }
        return false;
    };
    // exhaustive order: the zmarch family first (small), then direct by index
    int64_t ex_fam = 0, ex_idx = 0;
    std::vector<int> ex_fams = fams;
    std::reverse(ex_fams.begin(), ex_fams.end());
    auto draw_exhaustive = [&](Config *c) {
        while (ex_fam < (int64_t)ex_fams.size()) {
            int fam = ex_fams[ex_fam];
            while (ex_idx < space_size(fam)) {
                int64_t idx = ex_idx++;
                if (valid_for(op, g, fam, idx, c) && !queued.count(config_string(*c))) return true;
            }
            ++ex_fam;
            ex_idx = 0;
        }
        return false;
    };
    // local search: neighbours of the best evaluated configuration
    auto index_of = [&](const Config &c, int64_t *idx) {
        std::vector<int> r = radices(c.family), dg;
        if (!config_digits(c, &dg)) return false;
        int64_t y = 0;
        for (size_t p = r.size(); p-- > 0;) y = y * r[p] + dg[p];
        *idx = y;
        return true;
    };
    std::vector<Eval> evals;
    for (auto &p : done) evals.push_back(p.second);
    auto best_so_far = [&]() -> const Eval * {
        const Eval *b = nullptr;
        for (auto &e : evals)
            if (e.ok && (!b || e.time_us < b->time_us)) b = &e;
        return b;
    };
    int random_phase = std::max(8, O.max_evals / 4);
    int produced = 0;
    // candidates compiling on host threads, in launch order
    struct Pending {
        Config cfg;
        std::string key;
        std::future<std::pair<kl_status, Compiled>> fut;
    };
    std::vector<Pending> pipe;

    // Bayesian optimisation (Sec. 5.3 tunes with it): after an initial random
    // design, the candidate of largest expected improvement of log(time) among
    // a pool of random unqueued configurations and the unqueued neighbours of
    // the five fastest so far; candidates still compiling count as observed at
    // their predicted value.  The surrogate's length scale is re-selected
    // after every 8 new observations.
    const int bo_initial = std::max(8, std::min(32, O.max_evals / 8));
    const int bo_pool = 512;
    const double bo_xi = 0.01;        // margin in log(time): about 1 %
    double bo_ls = 0;
    size_t bo_ls_n = 0;
    auto propose_bayes = [&](Config *c) -> bool {
        std::vector<double> X, y, P, C, f(kFeatDims);
        std::vector<std::pair<double, Config>> obs;
        for (auto &e : evals) {
            Config ec;
            std::string err;
            if (!e.ok || !(e.time_us > 0) || !std::isfinite(e.time_us)) continue;
            if (!config_parse(e.config, &ec, &err) || !config_features(ec, f.data())) continue;
            X.insert(X.end(), f.begin(), f.end());
            y.push_back(std::log(e.time_us));
            obs.emplace_back(e.time_us, ec);
        }
        int n = (int)y.size();
        if (n < 2) return false;
        for (auto &p : pipe)
            if (config_features(p.cfg, f.data())) P.insert(P.end(), f.begin(), f.end());
        std::vector<Config> pool;
        std::set<std::string> in_pool;
        auto add = [&](const Config &k) {
            std::string s = config_string(k);
            if (queued.count(s) || !config_features(k, f.data()) || !in_pool.insert(s).second) return;
            pool.push_back(k);
            C.insert(C.end(), f.begin(), f.end());
        };
        std::sort(obs.begin(), obs.end(), [](const std::pair<double, Config> &a,
                                             const std::pair<double, Config> &b) { return a.first < b.first; });
        for (size_t q = 0; q < obs.size() && q < 5; ++q) {
            int64_t idx;
            if (!index_of(obs[q].second, &idx)) continue;
            for (int64_t nb : neighbours(obs[q].second.family, idx)) {
                Config k;
                if (valid_for(op, g, obs[q].second.family, nb, &k)) add(k);
            }
        }
        for (int q = 0; q < bo_pool; ++q) {
            Config k;
            if (!draw_random(&k)) break;
            add(k);
        }
        if (pool.empty()) return false;
        double ls = bo_ls > 0 && (size_t)n < bo_ls_n + 8 ? bo_ls : 0.0, used = 0;
        std::vector<double> ei;
        std::string err;
        int pick = bo_suggest(n, kFeatDims, X.data(), y.data(), (int)(P.size() / kFeatDims), P.data(),
                              (int)pool.size(), C.data(), bo_xi, ls, 0.0, &used, &ei, &err);
        if (pick < 0) return false;
        if (ls <= 0) {
            bo_ls = used;
            bo_ls_n = (size_t)n;
        }
        *c = pool[pick];
        return true;
    };

    auto next_candidate = [&](Config *c) -> bool {
        if (O.strategy == "exhaustive") return draw_exhaustive(c);
        if (O.strategy == "bayes" && produced >= bo_initial && propose_bayes(c)) return true;
        if (O.strategy == "local" && produced >= random_phase) {
            const Eval *b = best_so_far();
            Config bc;
            std::string err;
            int64_t idx;
            if (b && config_parse(b->config, &bc, &err) && index_of(bc, &idx)) {
                std::vector<int64_t> nb = neighbours(bc.family, idx);
                std::shuffle(nb.begin(), nb.end(), rng);
                for (int64_t n : nb)
                    if (valid_for(op, g, bc.family, n, c) && !queued.count(config_string(*c)))
                        return true;
            }
        }
        return draw_random(c);
    };

    // compile ahead on host threads (NVRTC only; modules load on this thread)
    int nthreads = O.threads > 0 ? O.threads
                   : std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
    int zuni = g.zh ? 0 : 1;
    auto launch_compile = [&](const Config &c) {
        Pending p;
        p.cfg = c;
        p.key = kernel_key(ctx, op, c, g.zbc, zuni);
        queued.insert(config_string(c));
        ++produced;
        std::string key = p.key;
        bool cached = ctx->kernels.count(key) > 0;
        p.fut = std::async(std::launch::async, [key, cached]() {
            Compiled out;
            kl_status s = cached ? KL_OK : nvrtc_compile(key, false, &out);
            return std::make_pair(s, std::move(out));
        });
        pipe.push_back(std::move(p));
    };
    int evaluated = (int)done.size();
    auto budget_left = [&]() { return elapsed() < O.budget_s && evaluated < O.max_evals; };
    while (budget_left() || !pipe.empty()) {
        while (budget_left() && (int)pipe.size() < nthreads) {
            Config c;
            if (!next_candidate(&c)) break;
            launch_compile(c);
            // keep the search adaptive: one new candidate per evaluation
            if (O.strategy == "local" && produced > random_phase) break;
            if (O.strategy == "bayes" && produced > bo_initial) break;
        }
        if (pipe.empty()) break;
        Pending p = std::move(pipe.front());
        pipe.erase(pipe.begin());
        auto res = p.fut.get();
        Eval e;
        e.config = config_string(p.cfg);
        if (!budget_left() && evaluated >= O.max_evals) {
            continue;   // drained after the budget: not evaluated
        }
        if (res.first != KL_OK) {
            e.note = "compile failed";
        } else {
            Kernel *k = nullptr;
            kl_status ls = ctx->kernels.count(p.key)
                               ? get_kernel(ctx, op, p.cfg, g.zbc, zuni, &k)
                               : load_compiled(ctx, op, p.cfg, p.key, res.second, &k);
            if (ls != KL_OK) {
                e.note = std::string("load failed: ") + kl_last_error();
                cudaGetLastError();
            } else if (reset_outputs(op, R) != KL_OK) {
                return KL_ERR_CUDA;
            } else {
                kl_status ts = time_config(ctx, op, p.cfg, g, R, 0, 1, &e.time_us);
                if (ts == KL_OK && op.accumulate) ts = reset_outputs(op, R);
                if (ts == KL_OK) ts = time_config(ctx, op, p.cfg, g, R, 0, 1, &e.time_us);
                if (ts == KL_OK && !op.accumulate) ts = verify(ctx, op, g, R, &e.err);
                if (ts == KL_OK && op.accumulate) {
                    // accumulate: verify one fresh application against the reference
                    reset_outputs(op, R);
                    kl_fields f{R.in[0], R.in[1], R.in[2], nin > 3 ? R.in[3] : nullptr, R.out[0], R.out[1], R.out[2]};
                    ts = launch_config(ctx, op, p.cfg, g, f, 0);
                    if (ts == KL_OK) ts = verify(ctx, op, g, R, &e.err);
                }
                if (ts == KL_OK && !op.accumulate)
                    ts = time_config(ctx, op, p.cfg, g, R, O.warm, O.reps, &e.time_us);
                if (ts != KL_OK) {
                    e.note = std::string("run failed: ") + kl_last_error();
                    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
                        return fail(KL_ERR_CUDA, "tune: device error, stopping: " + e.note);
                } else {
                    e.ok = e.err <= tol;
                    if (!e.ok) e.note = "verification failed";
                }
            }
        }
        ++evaluated;
        evals.push_back(e);
        log_eval(O.log, e, elapsed());
    }

    // re-time the top candidates and the default
    std::vector<Eval> ok;
    for (auto &e : evals)
        if (e.ok) ok.push_back(e);
    std::sort(ok.begin(), ok.end(), [](const Eval &a, const Eval &b) { return a.time_us < b.time_us; });
    if (ok.size() > (size_t)O.topk) ok.resize(O.topk);
    double def_us = INFINITY;
    if (!op.accumulate) {
        st = time_config(ctx, op, def, g, R, O.warm, 3 * O.reps, &def_us);
        if (st) return st;
    }
    Eval best;
    best.config = config_string(def);
    best.time_us = def_us;
    best.ok = true;
    for (auto &e : ok) {
        Config c;
        std::string err;
        if (!config_parse(e.config, &c, &err)) continue;
        double t = e.time_us;
        if (!op.accumulate) {
            st = time_config(ctx, op, c, g, R, O.warm, 3 * O.reps, &t);
            if (st) return st;
        }
        if (t < best.time_us) {
            best = e;
            best.time_us = t;
        }
    }

    WisdomRecord rec;
    rec.device = ctx->name;
    rec.cc_major = ctx->cc_major;
    rec.cc_minor = ctx->cc_minor;
    rec.zbc = g.zbc;
    rec.nx = g.nx;
    rec.ny = g.ny;
    rec.nz = g.nz;
    rec.config = best.config;
    rec.time_us = best.time_us;
    int dv = 0, rv = 0, nvM = 0, nvm = 0;
    cudaDriverGetVersion(&dv);
    cudaRuntimeGetVersion(&rv);
    nvrtcVersion(&nvM, &nvm);
    char buf[64];
    rec.extra["date"] = now_iso();
    rec.extra["host"] = host_name();
    rec.extra["driver"] = std::to_string(dv);
    rec.extra["runtime"] = std::to_string(rv);
    snprintf(buf, sizeof buf, "%d.%d", nvM, nvm);
    rec.extra["nvrtc"] = buf;
    rec.extra["sms"] = std::to_string(ctx->nsm);
    rec.extra["strategy"] = O.strategy;
    rec.extra["family"] = O.family;
    rec.extra["evals"] = std::to_string(evaluated);
    snprintf(buf, sizeof buf, "%.1f", elapsed());
    rec.extra["tune_s"] = buf;
    snprintf(buf, sizeof buf, "%.3f", def_us);
    rec.extra["default_us"] = buf;
    snprintf(buf, sizeof buf, "%.3f", std::isfinite(def_us) && best.time_us > 0 ? def_us / best.time_us : 1.0);
    rec.extra["speedup"] = buf;
    rec.extra["dtype"] = dtype_tag(op.dtype);
    rec.extra["zuni"] = std::to_string(zuni);
    std::string err;
    if (!wisdom_append(wisdom_path, rec, &err)) return fail(KL_ERR_IO, err);
    return KL_OK;
}

kl_status kl_batch_shard(int32_t n, const int64_t *points, int32_t world, int32_t rank,
                         int32_t *out, int32_t *count, int64_t *load)
{
    if (n < 0 || world < 1 || rank < 0 || rank >= world || (n > 0 && (!points || !out)) || !count)
        return fail(KL_ERR_INVALID_ARG, "batch shard: bad arguments");
    for (int32_t q = 0; q < n; ++q)
        if (points[q] < 0) return fail(KL_ERR_INVALID_ARG, "batch shard: negative point count");
    // longest processing time first: grids by points, largest first (ties by
    // index), each to the rank with the least load so far (ties to the lower
    // rank).  Every rank computes the same assignment without communication.
    std::vector<int32_t> order((size_t)n);
    for (int32_t q = 0; q < n; ++q) order[(size_t)q] = q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return points[a] > points[b]; });
    std::vector<int64_t> loads((size_t)world, 0);
    std::vector<int32_t> owner((size_t)n);
    for (int32_t q : order) {
        int32_t r = (int32_t)(std::min_element(loads.begin(), loads.end()) - loads.begin());
        owner[(size_t)q] = r;
        loads[(size_t)r] += points[q];
    }
    int32_t m = 0;
    for (int32_t q = 0; q < n; ++q)
        if (owner[(size_t)q] == rank) out[m++] = q;       // ascending grid index
    *count = m;
    if (load) *load = loads[(size_t)rank];
    return KL_OK;
}

kl_status kl_launch_batched(kl_ctx *ctx, const kl_op *op, int32_t n, const kl_grid *grids,
                            const kl_fields *fields, void *stream)
{
    if (!ctx || !grids || !fields) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    if (n < 1) return fail(KL_ERR_INVALID_ARG, "batch needs at least one grid");
    kl_status st = check_op(op);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // the batch's identity: op, every grid (with its z profile) and every
    // field pointer.  A batch seen before replays the CUDA graph that holds
    // all of its launches (one graph launch), unless the caller's stream is
    // itself being captured, in which case the launches go into that capture.
    uint64_t bh = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t nb) {
        const unsigned char *c = (const unsigned char *)p;
        for (size_t q = 0; q < nb; ++q) bh = (bh ^ c[q]) * 1099511628211ull;
    };
    mix(op, sizeof *op);
    mix(&n, sizeof n);
    for (int i = 0; i < n; ++i) {
        mix(&grids[i], offsetof(kl_grid, zh));
        mix(&fields[i], sizeof fields[i]);
        if (grids[i].zh && grids[i].nz > 0) mix(grids[i].zh, sizeof(double) * ((size_t)grids[i].nz + 1));
    }
    const std::string bkey = "graph:" + std::to_string(bh) + ":" + std::to_string(n);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return fail(KL_ERR_CUDA, "batch: stream query");
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (!capturing) {
        auto gi = ctx->graphs.find(bkey);
        if (gi != ctx->graphs.end()) {
            if (cudaGraphLaunch(gi->second, s) != cudaSuccess) return fail(KL_ERR_CUDA, "batch graph launch");
            ctx->graph_replays++;
            return KL_OK;
        }
    }

    // the batch's configuration: the record tuned for the problem size
    // nearest to the batch's total point count (per boundary kind), for
    // every grid it fits; a grid it does not fit takes the record of its own
    // nearest tuned size (Sec. 4.5 rules)
    struct Item {
        Config cfg;
        KArgs a;
        CUtensorMap maps[KL_NMAPS];
    };
    std::vector<Item> items((size_t)n);
    std::map<std::string, std::vector<int>> groups;       // compile key -> grids
    long long points[2] = {0, 0};
    for (int i = 0; i < n; ++i) {
        st = check_fields(*op, &fields[i]);
        if (st) return fail(st, "grid " + std::to_string(i) + ": " + kl_last_error());
        st = check_grid(&grids[i], halo_of(*op), nullptr);
        if (st) return fail(st, "grid " + std::to_string(i) + ": " + kl_last_error());
        points[grids[i].zbc] += (long long)grids[i].nx * grids[i].ny * grids[i].nz;
    }
    Config bcfg[2];
    for (int z = 0; z < 2; ++z)
        if (points[z]) {
            st = select_batch_config(ctx, *op, z, points[z], &bcfg[z]);
            if (st) return st;
        }
    for (int i = 0; i < n; ++i) {
        Config cfg = bcfg[grids[i].zbc];
        std::string err0;
        if (!config_fits(*op, cfg, grids[i], &fields[i], &err0)) {
            st = select_config(ctx, *op, grids[i], &cfg);
            if (st) return st;
        }
        // a batch runs z chunks from its tile table, never persistent CTAs
        // (persistent CTAs over a class's tiles, in equal ranges that cross
        // from one grid to the next, measured slower than chunks that the
        // block scheduler balances); a record tuned with pe=1 or 2 (whose
        // launches ignore kc) takes chunks of at most 32 levels here
        if (cfg.family == 2 && cfg.pe) {
            cfg.pe = 0;
            cfg.kc = std::min(cfg.kc, 32);
        }
        std::string err;
        if (!config_fits(*op, cfg, grids[i], &fields[i], &err)) cfg = Config();
        items[i].cfg = cfg;
        st = make_kargs(ctx, *op, cfg, grids[i], fields[i], &items[i].a, items[i].maps);
        if (st) return fail(st, "grid " + std::to_string(i) + ": " + kl_last_error());
        int zuni = grids[i].zh ? 0 : 1;
        groups[compile_defines(*op, cfg, grids[i].zbc, zuni)].push_back(i);
    }

    ctx->last_batch.clear();
    for (auto &gp : groups)
        ctx->last_batch += (ctx->last_batch.empty() ? "" : "; ") + config_string(items[gp.second[0]].cfg) +
                           " x" + std::to_string(gp.second.size());
    // per configuration class: its device table [descriptors | argument
    // blocks | tile list] (uploaded once per content) and its compiled kernel
    struct Launch {
        Kernel *k;
        Config cfg;
        size_t nblocks;
        void *argv, *tl, *tm;
    };
    std::vector<Launch> plan;
    for (auto &gp : groups) {
        const std::vector<int> &ids = gp.second;
        const Config &cfg = items[ids[0]].cfg;
        const kl_grid &g0 = grids[ids[0]];
        std::vector<int> tiles;                 // 4 ints per block
        for (size_t q = 0; q < ids.size(); ++q) {
            const KArgs &a = items[ids[q]].a;
            if (cfg.family == 0) {
                long long nb = a.nbx * a.nby * a.nbz;
                for (long long b = 0; b < nb; ++b) {
                    tiles.push_back((int)q);
                    tiles.push_back((int)b);
                    tiles.push_back(0);
                    tiles.push_back(0);
                }
            } else {
                for (int bz = 0; bz < (int)a.nbz; ++bz)
                    for (int by = 0; by < (int)a.nby; ++by)
                        for (int bx = 0; bx < (int)a.nbx; ++bx) {
                            tiles.push_back((int)q);
                            tiles.push_back(bx);
                            tiles.push_back(by);
                            tiles.push_back(bz);
                        }
            }
        }
        size_t nblocks = tiles.size() / 4;
        if (nblocks == 0 || nblocks > 0x7fffffffULL) return fail(KL_ERR_UNSUPPORTED, "batch too large");
        size_t off_maps = 0, sz_maps = ids.size() * KL_NMAPS * sizeof(CUtensorMap);
        size_t off_args = (sz_maps + 63) / 64 * 64, sz_args = ids.size() * sizeof(KArgs);
        size_t off_tiles = (off_args + sz_args + 63) / 64 * 64;
        size_t total = off_tiles + tiles.size() * sizeof(int);
        std::vector<char> img(total, 0);
        for (size_t q = 0; q < ids.size(); ++q) {
            memcpy(img.data() + off_maps + q * KL_NMAPS * sizeof(CUtensorMap), items[ids[q]].maps,
                   KL_NMAPS * sizeof(CUtensorMap));
            memcpy(img.data() + off_args + q * sizeof(KArgs), &items[ids[q]].a, sizeof(KArgs));
        }
        memcpy(img.data() + off_tiles, tiles.data(), tiles.size() * sizeof(int));
        uint64_t h = 1469598103934665603ull;
        for (char c : gp.first) h = (h ^ (unsigned char)c) * 1099511628211ull;
        for (char c : img) h = (h ^ (unsigned char)c) * 1099511628211ull;
        std::string tkey = "batch:" + std::to_string(h) + ":" + std::to_string(total);
        auto it = ctx->tables.find(tkey);
        void *dev = nullptr;
        if (it != ctx->tables.end()) {
            dev = it->second.first;
        } else {
            if (ctx->tables.size() > 64) {              // bound the cache (graphs use tables)
                if (capturing) return fail(KL_ERR_UNSUPPORTED, "batch table cache full while capturing");
                cudaStreamSynchronize(s);
                for (cudaStream_t st2 : ctx->aux_streams) cudaStreamSynchronize(st2);
                for (auto &gr : ctx->graphs) cudaGraphExecDestroy(gr.second);
                ctx->graphs.clear();
                for (auto &t : ctx->tables) cudaFree(t.second.first);
                ctx->tables.clear();
            }
            if (capturing) return fail(KL_ERR_UNSUPPORTED, "a new batch cannot upload its table while the stream is captured");
            if (cudaMalloc(&dev, total) != cudaSuccess) return fail(KL_ERR_OOM, "batch table allocation");
            cudaError_t e = cudaMemcpy(dev, img.data(), total, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(dev);
                return cuda_fail(e, "batch table upload");
            }
            ctx->tables[tkey] = {dev, total};
        }
        Kernel *k = nullptr;
        st = get_kernel(ctx, *op, cfg, g0.zbc, g0.zh ? 0 : 1, &k, true);
        if (st) return st;
        char *base = (char *)dev;
        plan.push_back({k, cfg, nblocks, base + off_args, base + off_tiles, base + off_maps});
    }

    // streams: with several configuration classes, the classes run side by
    // side on up to kBatchStreams streams forked from s and joined back
    constexpr int kBatchStreams = 4;
    const int naux = plan.size() > 1 ? (int)std::min<size_t>(plan.size(), kBatchStreams) : 0;
    while ((int)ctx->aux_streams.size() < naux) {
        cudaStream_t st2;
        if (cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking) != cudaSuccess)
            return fail(KL_ERR_CUDA, "batch stream creation");
        ctx->aux_streams.push_back(st2);
    }
    while ((int)ctx->aux_events.size() < 1 + naux) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return fail(KL_ERR_CUDA, "batch event creation");
        ctx->aux_events.push_back(ev);
    }
    // all launches of the batch, forked from and joined back into `root`
    auto issue_all = [&](cudaStream_t root) -> kl_status {
        if (naux) {
            if (cudaEventRecord(ctx->aux_events[0], root) != cudaSuccess) return fail(KL_ERR_CUDA, "batch fork");
            for (int i = 0; i < naux; ++i)
                if (cudaStreamWaitEvent(ctx->aux_streams[i], ctx->aux_events[0], 0) != cudaSuccess)
                    return fail(KL_ERR_CUDA, "batch fork");
        }
        for (size_t q = 0; q < plan.size(); ++q) {
            const Launch &L = plan[q];
            cudaStream_t ls = naux ? ctx->aux_streams[q % naux] : root;
            void *argv = L.argv, *tl = L.tl, *tm = L.tm;
            CUresult r;
            if (L.cfg.family == 0) {
                void *params[] = {&argv, &tl};
                r = ctx->drv.LaunchKernel(L.k->fn, (unsigned)L.nblocks, 1, 1, L.cfg.bx, L.cfg.by,
                                          L.cfg.bz, 0, (CUstream)ls, params, nullptr);
            } else {
                void *params[] = {&argv, &tl, &tm};
                r = ctx->drv.LaunchKernel(L.k->fn, (unsigned)L.nblocks, 1, 1, L.cfg.mbx,
                                          zmarch_block_y(L.cfg), 1, (unsigned)L.k->smem, (CUstream)ls,
                                          params, nullptr);
            }
            if (r != CUDA_SUCCESS) return cu_fail(r, "cuLaunchKernel (batch)");
            ctx->launches++;
        }
        for (int i = 0; i < naux; ++i) {
            if (cudaEventRecord(ctx->aux_events[1 + i], ctx->aux_streams[i]) != cudaSuccess ||
                cudaStreamWaitEvent(root, ctx->aux_events[1 + i], 0) != cudaSuccess)
                return fail(KL_ERR_CUDA, "batch join");
        }
        return KL_OK;
    };
    if (capturing) return issue_all(s);

    // capture the launches into a graph once (on a private stream: capture
    // records, it runs nothing), then launch the graph on s, now and on every
    // repeat of the batch
    if (ctx->graphs.size() >= 16) {
        cudaStreamSynchronize(s);
        for (auto &gr : ctx->graphs) cudaGraphExecDestroy(gr.second);
        ctx->graphs.clear();
    }
    if (!ctx->cap_stream &&
        cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(KL_ERR_CUDA, "batch: capture stream creation");
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(KL_ERR_CUDA, "batch: begin capture");
    kl_status ist = issue_all(ctx->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (ist) {
        if (graph) cudaGraphDestroy(graph);
        return ist;
    }
    if (e != cudaSuccess || !graph) return cuda_fail(e, "batch: end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "batch: graph instantiate");
    ctx->graphs[bkey] = exec;
    if (cudaGraphLaunch(exec, s) != cudaSuccess) return fail(KL_ERR_CUDA, "batch graph launch");
    return KL_OK;
}

}  // extern "C"
