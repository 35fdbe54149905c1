// kl_api.cpp -- contexts, run-time compilation and module cache, launches,
// ghost fill and diagnostics entry points of the C ABI.
#include <nvrtc.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <sstream>
#include <thread>

#include <sys/stat.h>
#include <unistd.h>

#include "kl_internal.h"

namespace {

thread_local std::string g_last_error = "no error";

// NVRTC source of the tendency kernels, embedded at build time.
const char *kSource =
#include "kl_source.inc"
    ;

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

bool env_lists(const char *var, const char *name)
{
    const char *v = getenv(var);
    if (!v) return false;
    std::stringstream ss(v);
    std::string item;
    while (std::getline(ss, item, ','))
        if (item == name || item == "*") return true;
    return false;
}

}  // namespace

namespace kl {

void set_error(const std::string &msg) { g_last_error = msg; }

kl_status fail(kl_status code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

kl_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(KL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                                 cudaGetErrorString(e) + ")");
}

kl_status cu_fail(CUresult r, const char *what)
{
    return fail(KL_ERR_CUDA, std::string(what) + ": CUresult " + std::to_string((int)r));
}

// ------------------------------------------------------------ driver API

kl_status driver_load(Driver *d)
{
    struct Sym {
        const char *name;
        void **slot;
    } syms[] = {
        {"cuModuleLoadData", (void **)&d->ModuleLoadData},
        {"cuModuleUnload", (void **)&d->ModuleUnload},
        {"cuModuleGetFunction", (void **)&d->ModuleGetFunction},
        {"cuLaunchKernel", (void **)&d->LaunchKernel},
        {"cuFuncSetAttribute", (void **)&d->FuncSetAttribute},
        {"cuOccupancyMaxActiveBlocksPerMultiprocessor",
         (void **)&d->OccupancyMaxActiveBlocksPerMultiprocessor},
        {"cuFuncGetAttribute", (void **)&d->FuncGetAttribute},
        {"cuTensorMapEncodeTiled", (void **)&d->TensorMapEncodeTiled},
    };
    for (auto &s : syms) {
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion(s.name, s.slot, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !*s.slot)
            return fail(KL_ERR_CUDA, std::string("driver entry point not found: ") + s.name);
    }
    return KL_OK;
}

// ------------------------------------------------------------- NVRTC

kl_status nvrtc_compile(const std::string &defines, bool verbose, Compiled *out)
{
    nvrtcProgram prog;
    nvrtcResult r = nvrtcCreateProgram(&prog, kSource, "kl_stencil.cu", 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS) return fail(KL_ERR_NVRTC, nvrtcGetErrorString(r));
    std::vector<std::string> opts = {"-arch=sm_103a", "-std=c++17", "-lineinfo"};
    if (verbose) opts.push_back("--ptxas-options=-v");
    std::stringstream ss(defines);
    std::string tok;
    while (ss >> tok) opts.push_back(tok);
    std::vector<const char *> cops;
    for (auto &o : opts) cops.push_back(o.c_str());
    r = nvrtcCompileProgram(prog, (int)cops.size(), cops.data());
    size_t logn = 0;
    nvrtcGetProgramLogSize(prog, &logn);
    out->log.assign(logn, '\0');
    if (logn) nvrtcGetProgramLog(prog, &out->log[0]);
    while (!out->log.empty() && out->log.back() == '\0') out->log.pop_back();
    if (r != NVRTC_SUCCESS) {
        nvrtcDestroyProgram(&prog);
        return fail(KL_ERR_NVRTC, std::string("NVRTC: ") + nvrtcGetErrorString(r) + "\n" +
                                      defines + "\n" + out->log);
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    out->cubin.resize(n);
    nvrtcGetCUBIN(prog, out->cubin.data());
    nvrtcDestroyProgram(&prog);
    return KL_OK;
}

// ------------------------------------------------- on-disk cubin cache
//
// One file per compiled variant, <dir>/kl_<16 hex digits>.cubin: the line
// "KLCUBIN1 <identity bytes> <symbol bytes> <cubin bytes> <cubin FNV-1a>\n",
// the identity, the kernel's symbol name, then the cubin.  The identity names
// everything the cubin depends on: the FNV-1a hash of the source, the NVRTC
// version, the target and the compile options; the file name is the FNV-1a
// hash of the identity.  A file whose identity differs (another source or
// compiler, a name collision), whose lengths or checksum do not match, is not
// used and is rewritten.  Writes go to a unique temporary name and are
// renamed into place, so a reader never sees a partial file and concurrent
// writers of one variant leave one whole copy.

uint64_t fnv1a(const void *p, size_t n, uint64_t h)
{
    const unsigned char *b = (const unsigned char *)p;
    for (size_t q = 0; q < n; ++q) h = (h ^ b[q]) * 1099511628211ull;
    return h;
}

std::string cache_identity(uint64_t source_hash, const std::string &options)
{
    int M = 0, m = 0;
    nvrtcVersion(&M, &m);
    char b[128];
    snprintf(b, sizeof b, "source=%016llx nvrtc=%d.%d arch=sm_103a options=",
             (unsigned long long)source_hash, M, m);
    return b + options;
}

static std::string stencil_identity(const std::string &defines)
{
    static const uint64_t src = fnv1a(kSource, strlen(kSource));
    return cache_identity(src, defines);
}

static std::string cache_path(const std::string &dir, const std::string &ident)
{
    char b[40];
    snprintf(b, sizeof b, "kl_%016llx.cubin", (unsigned long long)fnv1a(ident.data(), ident.size()));
    return dir + "/" + b;
}

bool cache_read(const std::string &dir, const std::string &ident, Compiled *out)
{
    FILE *f = fopen(cache_path(dir, ident).c_str(), "rb");
    if (!f) return false;
    bool ok = false;
    char head[128];
    size_t ni = 0, ns = 0, nc = 0;
    unsigned long long sum = 0;
    if (fgets(head, sizeof head, f) &&
        sscanf(head, "KLCUBIN1 %zu %zu %zu %llx", &ni, &ns, &nc, &sum) == 4 && ni == ident.size() &&
        ns < 4096 && nc > 0 && nc < ((size_t)1 << 30)) {
        std::string id(ni, '\0'), sym(ns, '\0');
        std::vector<char> cubin(nc);
        char extra;
        if (fread(&id[0], 1, ni, f) == ni && id == ident && fread(&sym[0], 1, ns, f) == ns &&
            fread(cubin.data(), 1, nc, f) == nc && fread(&extra, 1, 1, f) == 0 &&
            fnv1a(cubin.data(), nc) == sum) {
            out->cubin.swap(cubin);
            out->symbol = sym;
            ok = true;
        }
    }
    fclose(f);
    return ok;
}

bool cache_write(const std::string &dir, const std::string &ident, const Compiled &c)
{
    std::string path = cache_path(dir, ident);
    std::string tmp = path + "." + std::to_string((long long)getpid()) + "." +
                      std::to_string(std::hash<std::thread::id>()(std::this_thread::get_id())) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return false;
    bool ok = fprintf(f, "KLCUBIN1 %zu %zu %zu %016llx\n", ident.size(), c.symbol.size(),
                      c.cubin.size(), (unsigned long long)fnv1a(c.cubin.data(), c.cubin.size())) > 0 &&
              fwrite(ident.data(), 1, ident.size(), f) == ident.size() &&
              fwrite(c.symbol.data(), 1, c.symbol.size(), f) == c.symbol.size() &&
              fwrite(c.cubin.data(), 1, c.cubin.size(), f) == c.cubin.size();
    ok = fclose(f) == 0 && ok;
    if (!ok || rename(tmp.c_str(), path.c_str()) != 0) {
        remove(tmp.c_str());
        return false;
    }
    return true;
}

// ------------------------------------------------------ kernel cache

kl_status load_compiled(kl_ctx *ctx, const kl_op &op, const Config &cfg, const std::string &key,
                        const Compiled &c, Kernel **out)
{
    auto it = ctx->kernels.find(key);
    if (it != ctx->kernels.end()) {
        *out = &it->second;
        return KL_OK;
    }
    auto t1 = std::chrono::steady_clock::now();
    Kernel k;
    k.cfg = cfg;
    CUresult r = ctx->drv.ModuleLoadData(&k.mod, c.cubin.data());
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuModuleLoadData");
    r = ctx->drv.ModuleGetFunction(&k.fn, k.mod, "kl_tendency");
    if (r != CUDA_SUCCESS) {
        ctx->drv.ModuleUnload(k.mod);
        return cu_fail(r, "cuModuleGetFunction");
    }
    ctx->drv.FuncGetAttribute(&k.nregs, CU_FUNC_ATTRIBUTE_NUM_REGS, k.fn);
    ctx->drv.FuncGetAttribute(&k.local_bytes, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, k.fn);
    if (cfg.family >= 1) {
        k.smem = zmarch_smem_bytes(op, cfg);
        r = ctx->drv.FuncSetAttribute(k.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                      (int)k.smem);
        if (r != CUDA_SUCCESS) {
            ctx->drv.ModuleUnload(k.mod);
            return cu_fail(r, "cuFuncSetAttribute(max dynamic smem)");
        }
    }
    ctx->t_load_ms += ms_since(t1);
    ctx->cache_misses++;
    auto ins = ctx->kernels.emplace(key, k);
    *out = &ins.first->second;
    return KL_OK;
}

std::string kernel_key(const kl_ctx *ctx, const kl_op &op, const Config &cfg, int zbc, int zuni)
{
    return compile_defines(op, cfg, zbc, zuni) +
           (ctx->wait_cycles != kDefaultWaitCycles ? " -DKL_WAITPOLL=1" : "");
}

kl_status get_kernel(kl_ctx *ctx, const kl_op &op, const Config &cfg, int zbc, int zuni,
                     Kernel **out, bool batch)
{
    std::string key = kernel_key(ctx, op, cfg, zbc, zuni) + (batch ? " -DKL_BATCH=1" : "");
    auto it = ctx->kernels.find(key);
    if (it != ctx->kernels.end()) {
        *out = &it->second;
        return KL_OK;
    }
    auto t0 = std::chrono::steady_clock::now();
    Compiled c;
    if (!ctx->cache_dir.empty() && cache_read(ctx->cache_dir, stencil_identity(key), &c)) {
        ctx->t_disk_ms += ms_since(t0);
        kl_status st = load_compiled(ctx, op, cfg, key, c, out);
        if (st == KL_OK) {
            ctx->disk_hits++;
            return KL_OK;
        }
        cudaGetLastError();   // an unusable file: compile it again below and replace it
        t0 = std::chrono::steady_clock::now();
    }
    kl_status st = nvrtc_compile(key, false, &c);
    if (st) return st;
    ctx->t_nvrtc_ms += ms_since(t0);
    if (!ctx->cache_dir.empty() && cache_write(ctx->cache_dir, stencil_identity(key), c))
        ctx->disk_writes++;
    return load_compiled(ctx, op, cfg, key, c, out);
}

// ----------------------------------------------------- z profiles

kl_status get_profile(kl_ctx *ctx, const kl_grid &g, Profile **out)
{
    // key: z grid description (content hash of zh, FNV-1a)
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t q = 0; q < n; ++q) h = (h ^ b[q]) * 1099511628211ull;
    };
    mix(&g.nz, sizeof g.nz);
    mix(&g.g, sizeof g.g);
    mix(&g.zbc, sizeof g.zbc);
    if (g.zh) mix(g.zh, sizeof(double) * (size_t)(g.nz + 1));
    else mix(&g.dz, sizeof g.dz);
    std::string key = std::to_string(h) + (g.zh ? "s" : "u");
    auto it = ctx->profiles.find(key);
    if (it != ctx->profiles.end()) {
        *out = &it->second;
        return KL_OK;
    }
    std::vector<double> dzi, dzhi;
    zprofile_host(g.nz, g.g, g.zbc, g.zh, g.dz, &dzi, &dzhi);
    int n = g.nz + 2 * g.g;
    // d64: dzi | dzhi | dz | dzh ; d32: dzi | dzhi
    std::vector<double> h64(4 * (size_t)n);
    std::vector<float> h32(2 * (size_t)n);
    for (int q = 0; q < n; ++q) {
        h64[q] = dzi[q];
        h64[n + q] = dzhi[q];
        h64[2 * n + q] = 1.0 / dzi[q];
        h64[3 * n + q] = 1.0 / dzhi[q];
        h32[q] = (float)dzi[q];
        h32[n + q] = (float)dzhi[q];
    }
    Profile p;
    p.n = n;
    cudaError_t e = cudaMalloc(&p.d64, sizeof(double) * h64.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(profile)");
    e = cudaMalloc(&p.d32, sizeof(float) * h32.size());
    if (e != cudaSuccess) {
        cudaFree(p.d64);
        return cuda_fail(e, "cudaMalloc(profile)");
    }
    e = cudaMemcpy(p.d64, h64.data(), sizeof(double) * h64.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p.d32, h32.data(), sizeof(float) * h32.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p.d64);
        cudaFree(p.d32);
        return cuda_fail(e, "cudaMemcpy(profile)");
    }
    auto ins = ctx->profiles.emplace(key, p);
    *out = &ins.first->second;
    return KL_OK;
}

// ------------------------------------------------------------ launch

kl_status check_op(const kl_op *op)
{
    if (!op) return fail(KL_ERR_INVALID_ARG, "op is NULL");
    if (op->adv != 0 && op->adv != 2 && op->adv != 5)
        return fail(KL_ERR_INVALID_ARG, "adv must be 0, 2 or 5");
    if (op->diff < 0 || op->diff > 2) return fail(KL_ERR_INVALID_ARG, "diff must be 0, 1 or 2");
    if (op->dtype < KL_F64 || op->dtype > KL_F16)
        return fail(KL_ERR_INVALID_ARG, "dtype must be 0..3");
    if (op->accumulate != 0 && op->accumulate != 1)
        return fail(KL_ERR_INVALID_ARG, "accumulate must be 0 or 1");
    if (op->out_f32 != 0 && op->out_f32 != 1)
        return fail(KL_ERR_INVALID_ARG, "out_f32 must be 0 or 1");
    if (op->out_f32 && op->dtype != KL_BF16 && op->dtype != KL_F16)
        return fail(KL_ERR_INVALID_ARG, "out_f32 applies to 16-bit storage (bf16, f16)");
    return KL_OK;
}

kl_status check_fields(const kl_op &op, const kl_fields *f)
{
    if (!f) return fail(KL_ERR_INVALID_ARG, "fields is NULL");
    if (!f->u || !f->v || !f->w || !f->ut || !f->vt || !f->wt)
        return fail(KL_ERR_INVALID_ARG, "a field pointer is NULL");
    if (op.diff == 2 && !f->nu) return fail(KL_ERR_INVALID_ARG, "diff = 2 needs the nu field");
    const uintptr_t es = (uintptr_t)esize_of(op.dtype), eo = (uintptr_t)esize_of(out_dtype(op));
    const void *ps[] = {f->u, f->v, f->w, op.diff == 2 ? f->nu : f->u};
    for (const void *p : ps)
        if ((uintptr_t)p % es) return fail(KL_ERR_INVALID_ARG, "misaligned field pointer");
    const void *po[] = {f->ut, f->vt, f->wt};
    for (const void *p : po)
        if ((uintptr_t)p % eo) return fail(KL_ERR_INVALID_ARG, "misaligned tendency pointer");
    return KL_OK;
}

static void fill_coefs(KArgs &a, const kl_grid &g)
{
    double dzi = g.zh ? 0.0 : 1.0 / g.dz;
    double c[8] = {1.0 / g.dx, 1.0 / g.dy, dzi, dzi, g.nu, g.nu / (g.dx * g.dx),
                   g.nu / (g.dy * g.dy), 0.0};
    for (int q = 0; q < 8; ++q) {
        a.cd[q] = c[q];
        a.cf[q] = (float)c[q];
    }
}

bool config_fits(const kl_op &op, const Config &cfg, const kl_grid &g, const kl_fields *f,
                 std::string *why)
{
    if (cfg.family == 0) return true;
    Geom geo;
    if (check_grid(&g, halo_of(op), &geo) != KL_OK) {
        *why = "grid invalid";
        return false;
    }
    int es = esize_of(op.dtype);
    if ((geo.x0 * es) % 16 || (g.sj * es) % 16 || (g.sk * es) % 16) {
        *why = "zmarch needs the interior x start and the strides 16-byte aligned";
        return false;
    }
    if (f) {
        const void *ps[4] = {f->u, f->v, f->w, op.diff == 2 ? f->nu : f->u};
        for (const void *p : ps)
            if ((uintptr_t)p % 16) {
                *why = "zmarch needs 16-byte aligned field pointers";
                return false;
            }
    }
    return true;
}

// TMA descriptor of one field for the zmarch box; cached by pointer and layout
// (box_x elements wide, z.rows rows, one plane)
static kl_status get_tmap(kl_ctx *ctx, const kl_op &op, const kl_grid &g, int box_x, int box_y,
                          const void *ptr, CUtensorMap *out)
{
    char key[256];
    snprintf(key, sizeof key, "%p/%d/%lld/%lld/%lld/%d/%d", ptr, op.dtype, (long long)g.sj,
             (long long)g.sk, (long long)g.extent, box_x, box_y);
    auto it = ctx->tmaps.find(key);
    if (it != ctx->tmaps.end()) {
        *out = it->second;
        return KL_OK;
    }
    int es = esize_of(op.dtype);
    CUtensorMapDataType dt = op.dtype == KL_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                             : op.dtype == KL_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                  : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    cuuint64_t dims[3] = {(cuuint64_t)g.sj, (cuuint64_t)(g.sk / g.sj), (cuuint64_t)(g.extent / g.sk)};
    cuuint64_t strides[2] = {(cuuint64_t)(g.sj * es), (cuuint64_t)(g.sk * es)};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    CUresult r = ctx->drv.TensorMapEncodeTiled(&m, dt, 3, const_cast<void *>(ptr), dims, strides, box,
                                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                               CU_TENSOR_MAP_SWIZZLE_NONE,
                                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuTensorMapEncodeTiled");
    if (ctx->tmaps.size() > 4096) ctx->tmaps.clear();
    ctx->tmaps[key] = m;
    *out = m;
    return KL_OK;
}

kl_status make_kargs(kl_ctx *ctx, const kl_op &op, const Config &cfg, const kl_grid &g,
                     const kl_fields &f, KArgs *ap, CUtensorMap maps[KL_NMAPS])
{
    std::string err;
    if (!config_check(op, cfg, &err)) return fail(KL_ERR_INVALID_ARG, "configuration: " + err);
    Geom geo;
    kl_status st = check_grid(&g, halo_of(op), &geo);
    if (st) return st;
    if (!config_fits(op, cfg, g, &f, &err)) return fail(KL_ERR_INVALID_ARG, "configuration: " + err);
    Profile *prof = nullptr;
    if (g.zh) {
        st = get_profile(ctx, g, &prof);
        if (st) return st;
    }
    int es = esize_of(op.dtype);
    KArgs &a = *ap;
    memset(&a, 0, sizeof a);
    const char *base[7] = {(const char *)f.u, (const char *)f.v, (const char *)f.w,
                           (const char *)f.nu, (const char *)f.ut, (const char *)f.vt,
                           (const char *)f.wt};
    size_t off = (size_t)g.origin * es;
    a.u = base[0] + off;
    a.v = base[1] + off;
    a.w = base[2] + off;
    a.nu = f.nu ? base[3] + off : nullptr;
    size_t offo = (size_t)g.origin * esize_of(out_dtype(op));
    a.ut = (void *)(base[4] + offo);
    a.vt = (void *)(base[5] + offo);
    a.wt = (void *)(base[6] + offo);
    if (prof) {
        if (op.dtype == KL_F64) {
            a.dzi = prof->d64 + g.g;
            a.dzhi = prof->d64 + prof->n + g.g;
        } else {
            a.dzi = prof->d32 + g.g;
            a.dzhi = prof->d32 + prof->n + g.g;
        }
    }
    a.err = ctx->d_err;
    a.wait_cycles = ctx->wait_cycles;
    a.flags = g.xybc ? 1 : 0;
    a.sj = g.sj;
    a.sk = g.sk;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.tile_x0 = geo.x0;
    a.tile_y0 = geo.y0;
    a.tile_z0 = geo.z0;
    fill_coefs(a, g);
    if (cfg.family == 0) {
        a.nbx = (g.nx + cfg.bx * cfg.tx - 1) / (cfg.bx * cfg.tx);
        a.nby = (g.ny + cfg.by * cfg.ty - 1) / (cfg.by * cfg.ty);
        a.nbz = (g.nz + cfg.bz * cfg.tz - 1) / (cfg.bz * cfg.tz);
    } else {
        ZGeom z = zmarch_geometry(op, cfg);
        a.kchunk = cfg.kc;
        a.nbx = (g.nx + z.txs - 1) / z.txs;
        a.nby = (g.ny + z.tys - 1) / z.tys;
        a.nbz = (g.nz + cfg.kc - 1) / cfg.kc;
        const void *fp[KL_NMAPS] = {f.u, f.v, f.w, op.diff == 2 ? f.nu : f.u, f.u, f.v, f.w};
        for (int q = 0; q < KL_NMAPS; ++q) {
            // zpack's x-wrap strips are 32 bytes wide; zmarch never reads maps 4..6;
            // zpack's nu box spans tile rows -1 .. tys
            int bx = q >= 4 && cfg.family == 2 ? 32 / es : z.pitch;
            int by = q == 3 && cfg.family == 2 ? z.tys + 2 : z.rows;
            st = get_tmap(ctx, op, g, bx, by, fp[q], &maps[q]);
            if (st) return st;
        }
    }
    return KL_OK;
}

kl_status launch_config(kl_ctx *ctx, const kl_op &op, const Config &cfg, const kl_grid &g,
                        const kl_fields &f, cudaStream_t s)
{
    KArgs a;
    CUtensorMap maps[KL_NMAPS];
    kl_status st = make_kargs(ctx, op, cfg, g, f, &a, maps);
    if (st) return st;
    if (!space_size(cfg.family)) return fail(KL_ERR_INVALID_ARG, "unknown family");
    int zuni = g.zh ? 0 : 1;
    Kernel *k = nullptr;
    auto t0 = std::chrono::steady_clock::now();
    bool miss = ctx->kernels.find(kernel_key(ctx, op, cfg, g.zbc, zuni)) == ctx->kernels.end();
    st = get_kernel(ctx, op, cfg, g.zbc, zuni, &k);
    if (st) return st;
    if (!miss) ctx->cache_hits++;

    CUresult r;
    auto t_launch = std::chrono::steady_clock::now();
    if (cfg.family == 0) {
        long long nb = a.nbx * a.nby * a.nbz;
        if (nb > 0x7fffffffLL) return fail(KL_ERR_UNSUPPORTED, "grid too large");
        void *params[] = {&a};
        r = ctx->drv.LaunchKernel(k->fn, (unsigned)nb, 1, 1, cfg.bx, cfg.by, cfg.bz, 0,
                                  (CUstream)s, params, nullptr);
    } else {
        if (a.nby > 65535 || a.nbz > 65535) return fail(KL_ERR_UNSUPPORTED, "grid too large");
        // zmarch takes the first four descriptors, zpack all seven
        void *params[] = {&a, &maps[0], &maps[1], &maps[2], &maps[3], &maps[4], &maps[5], &maps[6]};
        unsigned gx = (unsigned)a.nbx, gy = (unsigned)a.nby, gz = (unsigned)a.nbz;
        if (cfg.family == 2 && cfg.pe) {
            // persistent: as many CTAs as fit on the device at once, each
            // taking an equal range of the (tile, level) pairs
            int per_sm = 0;
            r = ctx->drv.OccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k->fn, cfg.mbx * zmarch_block_y(cfg), k->smem);
            if (r != CUDA_SUCCESS) return cu_fail(r, "cuOccupancyMaxActiveBlocksPerMultiprocessor");
            const long long pairs = a.nbx * a.nby * g.nz;
            gx = (unsigned)std::max(1LL, std::min<long long>(pairs, (long long)std::max(1, per_sm) * ctx->nsm));
            gy = gz = 1;
        }
        r = ctx->drv.LaunchKernel(k->fn, gx, gy, gz, cfg.mbx, zmarch_block_y(cfg), 1, (unsigned)k->smem,
                                  (CUstream)s, params, nullptr);
    }
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuLaunchKernel");
    if (miss) ctx->t_launch_ms += ms_since(t_launch);
    (void)t0;
    ctx->launches++;
    ctx->last_config = config_string(cfg);
    return KL_OK;
}

kl_status select_config(kl_ctx *ctx, const kl_op &op, const kl_grid &g, Config *cfg)
{
    char key[160];
    snprintf(key, sizeof key, "%d/%d/%d/%d/%d/%d/%d/%d", op.adv, op.diff, op.dtype,
             op.accumulate, g.zbc, g.nx, g.ny, g.nz);
    auto it = ctx->selection.find(key);
    std::string text;
    if (it != ctx->selection.end()) {
        text = it->second;
    } else {
        auto t0 = std::chrono::steady_clock::now();
        std::vector<WisdomRecord> recs;
        std::string err;
        int rule = 5;
        text = "default";
        if (!ctx->wisdom_dir.empty()) {
            std::string path = ctx->wisdom_dir + "/" + wisdom_file_name(op);
            if (wisdom_read(path, &recs, &err))
                rule = wisdom_select(recs, ctx->name, ctx->cc_major, ctx->cc_minor, g.zbc, g.nx,
                                     g.ny, g.nz, &text);
            else
                ctx->last_rule_text = err;
        }
        // a record whose configuration is invalid here falls back to the default
        Config c;
        if (!config_parse(text, &c, &err) || !config_check(op, c, &err) ||
            !config_fits(op, c, g, nullptr, &err)) {
            ctx->last_rule_text = "wisdom config rejected (" + err + "); default used";
            text = "default";
            rule = 5;
        }
        ctx->selection[key] = text;
        ctx->selection_rule[key] = rule;
        ctx->t_wisdom_ms += ms_since(t0);
    }
    std::string err;
    if (!config_parse(text, cfg, &err)) return fail(KL_ERR_WISDOM_PARSE, err);
    return KL_OK;
}

kl_status select_batch_config(kl_ctx *ctx, const kl_op &op, int zbc, long long points, Config *cfg)
{
    char key[160];
    snprintf(key, sizeof key, "batch/%d/%d/%d/%d/%d/%lld", op.adv, op.diff, op.dtype, op.accumulate,
             zbc, points);
    auto it = ctx->selection.find(key);
    std::string text;
    if (it != ctx->selection.end()) {
        text = it->second;
    } else {
        auto t0 = std::chrono::steady_clock::now();
        std::vector<WisdomRecord> recs;
        std::string err;
        int rule = 5;
        text = "default";
        if (!ctx->wisdom_dir.empty()) {
            std::string path = ctx->wisdom_dir + "/" + wisdom_file_name(op);
            if (wisdom_read(path, &recs, &err))
                rule = wisdom_select_points(recs, ctx->name, ctx->cc_major, ctx->cc_minor, zbc,
                                            (double)points, &text);
            else
                ctx->last_rule_text = err;
        }
        Config c;
        if (!config_parse(text, &c, &err) || !config_check(op, c, &err)) {
            text = "default";
            rule = 5;
        }
        ctx->selection[key] = text;
        ctx->selection_rule[key] = rule;
        ctx->t_wisdom_ms += ms_since(t0);
    }
    std::string err;
    if (!config_parse(text, cfg, &err)) return fail(KL_ERR_WISDOM_PARSE, err);
    return KL_OK;
}

}  // namespace kl

using namespace kl;

// ================================================================= C ABI

extern "C" {

const char *kl_last_error(void) { return g_last_error.c_str(); }

const char *kl_version(void) { return "libkl 0.1 (sm_103a, NVRTC)"; }

kl_status kl_create(kl_ctx **out, int device, const char *wisdom_dir)
{
    if (!out) return fail(KL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(KL_ERR_INVALID_ARG, "no such device");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    e = cudaFree(nullptr);  // make the primary context current on this thread
    if (e != cudaSuccess) return cuda_fail(e, "context init");
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    kl_ctx *c = new kl_ctx();
    c->device = device;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    c->nsm = prop.multiProcessorCount;
    c->name = prop.name;
    if (wisdom_dir) c->wisdom_dir = wisdom_dir;
    else if (const char *w = getenv("KL_WISDOM_DIR")) c->wisdom_dir = w;
    if (const char *cd = getenv("KL_CACHE_DIR")) c->cache_dir = cd;
    kl_status st = driver_load(&c->drv);
    if (st) {
        delete c;
        return st;
    }
    e = cudaMalloc(&c->d_err, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_out, sizeof(double) * 8);
    if (e != cudaSuccess) {
        kl_destroy(c);
        return cuda_fail(e, "context buffers");
    }
    *out = c;
    return KL_OK;
}

void kl_destroy(kl_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &p : c->kernels)
        if (p.second.mod) c->drv.ModuleUnload(p.second.mod);
    def_kernels_unload(c);
    for (auto &p : c->profiles) {
        cudaFree(p.second.d64);
        cudaFree(p.second.d32);
    }
    for (auto &p : c->tables) cudaFree(p.second.first);
    for (auto &gr : c->graphs) cudaGraphExecDestroy(gr.second);
    for (cudaStream_t st : c->aux_streams) cudaStreamDestroy(st);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t ev : c->aux_events) cudaEventDestroy(ev);
    cudaFree(c->d_err);
    cudaFree(c->d_scratch);
    if (c->h_out) cudaFreeHost(c->h_out);
    delete c;
}

kl_status kl_layout(int32_t nx, int32_t ny, int32_t nz, int32_t g, int32_t dtype, int64_t *sj,
                    int64_t *sk, int64_t *origin, int64_t *extent)
{
    if (nx < 1 || ny < 1 || nz < 1 || g < 0 || dtype < 0 || dtype > 3 || !sj || !sk || !origin ||
        !extent)
        return fail(KL_ERR_INVALID_ARG, "kl_layout: bad argument");
    int64_t al = 128 / esize_of(dtype);                 // elements per 128 bytes
    int64_t x0 = (g + al - 1) / al * al;                // interior x start, aligned
    int64_t row = (x0 + nx + g + al - 1) / al * al;     // row pitch, aligned
    *sj = row;
    *sk = row * (ny + 2 * (int64_t)g);
    *origin = x0 + (int64_t)g * *sj + (int64_t)g * *sk;
    *extent = *sk * (nz + 2 * (int64_t)g);
    if (*extent >= (int64_t(1) << 31)) return fail(KL_ERR_BOUNDS, "field larger than 2^31 elements");
    return KL_OK;
}

kl_status kl_fill_ghosts(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, void *u, void *v,
                         void *w, void *nu, void *stream)
{
    if (!ctx) return fail(KL_ERR_INVALID_ARG, "ctx is NULL");
    if (dtype < 0 || dtype > 3) return fail(KL_ERR_INVALID_ARG, "dtype must be 0..3");
    kl_status st = check_grid(grid, 1, nullptr);
    if (st) return st;
    if (!u || !v || !w) return fail(KL_ERR_INVALID_ARG, "u, v, w must not be NULL");
    if (grid->g > 4) return fail(KL_ERR_UNSUPPORTED, "ghost fill supports g <= 4");
    cudaError_t e = fill_ghosts_launch(esize_of(dtype), *grid, u, v, w, nu, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fill ghosts launch");
    ctx->launches++;
    return KL_OK;
}


// ------------------------------------------------------- halo strips

// one strided copy between a contiguous host array and the interior of a
// padded device field: cudaMemcpy3DAsync when the plane pitch is a whole
// number of rows, else one 2D copy per level
static kl_status copy_interior(int32_t dtype, const kl_grid *grid, const void *host, void *dev,
                               bool in, void *stream)
{
    if (!host || !dev) return fail(KL_ERR_INVALID_ARG, "host and dev must not be NULL");
    if (dtype < 0 || dtype > 3) return fail(KL_ERR_INVALID_ARG, "dtype must be 0..3");
    kl_status st = check_grid(grid, 0, nullptr);
    if (st) return st;
    const size_t es = (size_t)esize_of(dtype);
    const kl_grid &g = *grid;
    char *d0 = (char *)dev + (size_t)g.origin * es;
    const size_t row = (size_t)g.nx * es;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (g.sk % g.sj == 0) {
        cudaMemcpy3DParms p = {};
        cudaPitchedPtr dp = make_cudaPitchedPtr(d0, (size_t)g.sj * es, row, (size_t)(g.sk / g.sj));
        cudaPitchedPtr hp = make_cudaPitchedPtr((void *)host, row, row, (size_t)g.ny);
        p.extent = make_cudaExtent(row, (size_t)g.ny, (size_t)g.nz);
        if (in) {
            p.srcPtr = hp;
            p.dstPtr = dp;
            p.kind = cudaMemcpyHostToDevice;
        } else {
            p.srcPtr = dp;
            p.dstPtr = hp;
            p.kind = cudaMemcpyDeviceToHost;
        }
        e = cudaMemcpy3DAsync(&p, s);
    } else {
        for (int k = 0; k < g.nz && e == cudaSuccess; ++k) {
            char *dk = d0 + (size_t)k * g.sk * es;
            char *hk = (char *)host + (size_t)k * g.ny * row;
            e = in ? cudaMemcpy2DAsync(dk, (size_t)g.sj * es, hk, row, row, (size_t)g.ny,
                                       cudaMemcpyHostToDevice, s)
                   : cudaMemcpy2DAsync(hk, row, dk, (size_t)g.sj * es, row, (size_t)g.ny,
                                       cudaMemcpyDeviceToHost, s);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, in ? "kl_copy_in" : "kl_copy_out");
    return KL_OK;
}

static kl_status halo_check(int32_t dtype, const kl_grid *grid, int32_t axis, int32_t side,
                            int32_t nf)
{
    if (dtype < 0 || dtype > 3) return fail(KL_ERR_INVALID_ARG, "dtype must be 0..3");
    if (axis != 0 && axis != 1) return fail(KL_ERR_INVALID_ARG, "axis must be 0 (x) or 1 (y)");
    if (side != 0 && side != 1) return fail(KL_ERR_INVALID_ARG, "side must be 0 or 1");
    if (nf < 1 || nf > 4) return fail(KL_ERR_INVALID_ARG, "nf must be 1..4");
    return check_grid(grid, 1, nullptr);
}

kl_status kl_copy_in(int32_t dtype, const kl_grid *grid, const void *host, void *dev, void *stream)
{
    return copy_interior(dtype, grid, host, dev, true, stream);
}

kl_status kl_copy_out(int32_t dtype, const kl_grid *grid, const void *dev, void *host, void *stream)
{
    return copy_interior(dtype, grid, host, (void *)dev, false, stream);
}

kl_status kl_halo_bytes(const kl_grid *grid, int32_t dtype, int32_t axis, int32_t nf,
                        int64_t *bytes)
{
    if (!bytes) return fail(KL_ERR_INVALID_ARG, "bytes is NULL");
    kl_status st = halo_check(dtype, grid, axis, 0, nf);
    if (st) return st;
    int w, h;
    halo_strip_shape(*grid, axis, &w, &h);
    *bytes = (int64_t)w * h * grid->nz * nf * esize_of(dtype);
    return KL_OK;
}

static kl_status halo_move(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t axis,
                           int32_t side, int32_t nf, void *const *fields, void *buf, bool unpack,
                           void *stream)
{
    if (!ctx || !fields || !buf) return fail(KL_ERR_INVALID_ARG, "ctx, fields and buf must not be NULL");
    kl_status st = halo_check(dtype, grid, axis, side, nf);
    if (st) return st;
    for (int f = 0; f < nf; ++f)
        if (!fields[f]) return fail(KL_ERR_INVALID_ARG, "a field pointer is NULL");
    cudaError_t e = halo_launch(esize_of(dtype), *grid, axis, side, nf, fields, buf, unpack,
                                (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, unpack ? "halo unpack launch" : "halo pack launch");
    ctx->launches++;
    return KL_OK;
}

kl_status kl_halo_pack(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t axis,
                       int32_t side, int32_t nf, const void *const *fields, void *buf,
                       void *stream)
{
    return halo_move(ctx, dtype, grid, axis, side, nf, (void *const *)fields, buf, false, stream);
}

kl_status kl_halo_unpack(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t axis,
                         int32_t side, int32_t nf, void *const *fields, const void *buf,
                         void *stream)
{
    return halo_move(ctx, dtype, grid, axis, side, nf, fields, (void *)buf, true, stream);
}

kl_status kl_capture_if_requested(kl_ctx *ctx, const kl_op *op, const kl_grid *grid,
                                  const kl_fields *fields, void *stream);

kl_status kl_launch(kl_ctx *ctx, const kl_op *op, const kl_grid *grid, const kl_fields *fields,
                    void *stream)
{
    if (!ctx) return fail(KL_ERR_INVALID_ARG, "ctx is NULL");
    kl_status st = check_op(op);
    if (st) return st;
    st = check_fields(*op, fields);
    if (st) return st;
    st = check_grid(grid, halo_of(*op), nullptr);
    if (st) return st;
    if (env_lists("KERNEL_LAUNCHER_CAPTURE", "tendency")) {
        st = kl_capture_if_requested(ctx, op, grid, fields, stream);
        if (st) return st;
    }
    Config cfg;
    st = select_config(ctx, *op, *grid, &cfg);
    if (st) return st;
    return launch_config(ctx, *op, cfg, *grid, *fields, (cudaStream_t)stream);
}

// checks, configuration selection and the ghost fill that configuration
// needs (the zpack family wraps x itself: no x ghosts of interior rows)
static kl_status fill_for_op(kl_ctx *ctx, const kl_op *op, const kl_grid *grid,
                             const kl_fields *fields, void *stream, Config *cfg)
{
    if (!ctx) return fail(KL_ERR_INVALID_ARG, "ctx is NULL");
    kl_status st = check_op(op);
    if (st) return st;
    st = check_fields(*op, fields);
    if (st) return st;
    st = check_grid(grid, halo_of(*op), nullptr);
    if (st) return st;
    if (grid->g > 4) return fail(KL_ERR_UNSUPPORTED, "ghost fill supports g <= 4");
    st = select_config(ctx, *op, *grid, cfg);
    if (st) return st;
    // the zpack kernel forms the x halo itself on grids with nx >= 64 + H
    // (constant nu)
    const bool x_ghosts = !(cfg->family == 2 && op->diff != 2 && grid->nx >= 64 + halo_of(*op)) &&
                          !grid->xybc;
    cudaError_t e = fill_ghosts_launch(esize_of(op->dtype), *grid, (void *)fields->u,
                                       (void *)fields->v, (void *)fields->w, (void *)fields->nu,
                                       (cudaStream_t)stream, x_ghosts);
    if (e != cudaSuccess) return cuda_fail(e, "fill ghosts launch");
    ctx->launches++;
    return KL_OK;
}

kl_status kl_fill_ghosts_op(kl_ctx *ctx, const kl_op *op, const kl_grid *grid,
                            const kl_fields *fields, void *stream)
{
    Config cfg;
    return fill_for_op(ctx, op, grid, fields, stream, &cfg);
}

kl_status kl_step(kl_ctx *ctx, const kl_op *op, const kl_grid *grid, const kl_fields *fields,
                  void *stream)
{
    Config cfg;
    kl_status st = fill_for_op(ctx, op, grid, fields, stream, &cfg);
    if (st) return st;
    if (env_lists("KERNEL_LAUNCHER_CAPTURE", "tendency")) {
        st = kl_capture_if_requested(ctx, op, grid, fields, stream);
        if (st) return st;
    }
    return launch_config(ctx, *op, cfg, *grid, *fields, (cudaStream_t)stream);
}

kl_status kl_launch_with_config(kl_ctx *ctx, const kl_op *op, const char *config,
                                const kl_grid *grid, const kl_fields *fields, void *stream)
{
    if (!ctx || !config) return fail(KL_ERR_INVALID_ARG, "ctx or config is NULL");
    kl_status st = check_op(op);
    if (st) return st;
    st = check_fields(*op, fields);
    if (st) return st;
    Config cfg;
    std::string err;
    if (!config_parse(config, &cfg, &err)) return fail(KL_ERR_INVALID_ARG, err);
    return launch_config(ctx, *op, cfg, *grid, *fields, (cudaStream_t)stream);
}

kl_status kl_diag(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t level, const void *t,
                  const double *ref, double out[6], void *stream)
{
    if (!ctx || !t || !out) return fail(KL_ERR_INVALID_ARG, "ctx, t and out must not be NULL");
    if (dtype < 0 || dtype > 3 || (level != 0 && level != 1))
        return fail(KL_ERR_INVALID_ARG, "bad dtype or level");
    kl_status st = check_grid(grid, 1, nullptr);
    if (st) return st;
    Profile *prof = nullptr;
    st = get_profile(ctx, *grid, &prof);
    if (st) return st;
    int nb = diag_blocks(ctx->nsm);
    size_t need = (size_t)nb * 6 + 8;
    if (ctx->scratch_doubles < need) {
        cudaFree(ctx->d_scratch);
        ctx->d_scratch = nullptr;
        ctx->scratch_doubles = 0;
        cudaError_t e = cudaMalloc(&ctx->d_scratch, need * sizeof(double));
        if (e != cudaSuccess) return fail(KL_ERR_OOM, "cudaMalloc(diag scratch) failed");
        ctx->scratch_doubles = need;
    }
    const double *wz = prof->d64 + (level == 0 ? 2 : 3) * prof->n + grid->g;
    double *dout = ctx->d_scratch + (size_t)nb * 6;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = diag_launch(dtype, *grid, level, t, ref, wz, ctx->d_scratch, nb, dout, s);
    if (e != cudaSuccess) return cuda_fail(e, "diag launch");
    e = cudaMemcpyAsync(ctx->h_out, dout, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "diag readback");
    memcpy(out, ctx->h_out, 6 * sizeof(double));
    ctx->launches += 2;
    return KL_OK;
}

kl_status kl_dot(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t level, const void *a,
                 const void *b, double *out, void *stream)
{
    if (!ctx || !a || !b || !out) return fail(KL_ERR_INVALID_ARG, "ctx, a, b and out must not be NULL");
    if (dtype < 0 || dtype > 3 || level < -1 || level > 1)
        return fail(KL_ERR_INVALID_ARG, "bad dtype or level");
    kl_status st = check_grid(grid, 1, nullptr);
    if (st) return st;
    const double *wz = nullptr;
    if (level >= 0) {
        Profile *prof = nullptr;
        st = get_profile(ctx, *grid, &prof);
        if (st) return st;
        wz = prof->d64 + (level == 0 ? 2 : 3) * prof->n + grid->g;
    }
    int nb = diag_blocks(ctx->nsm);
    size_t need = (size_t)nb * 6 + 8;
    if (ctx->scratch_doubles < need) {
        cudaFree(ctx->d_scratch);
        ctx->d_scratch = nullptr;
        ctx->scratch_doubles = 0;
        cudaError_t e = cudaMalloc(&ctx->d_scratch, need * sizeof(double));
        if (e != cudaSuccess) return fail(KL_ERR_OOM, "cudaMalloc(diag scratch) failed");
        ctx->scratch_doubles = need;
    }
    double *dout = ctx->d_scratch + (size_t)nb * 6;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = dot_launch(dtype, *grid, a, b, wz, ctx->d_scratch, nb, dout, s);
    if (e != cudaSuccess) return cuda_fail(e, "dot launch");
    e = cudaMemcpyAsync(ctx->h_out, dout, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "dot readback");
    *out = ctx->h_out[4];
    ctx->launches += 2;
    return KL_OK;
}

kl_status kl_smagorinsky(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, double cs,
                         const void *u, const void *v, const void *w, void *nu,
                         int32_t fill_ghosts, void *stream)
{
    if (!ctx || !u || !v || !w || !nu) return fail(KL_ERR_INVALID_ARG, "ctx, u, v, w and nu must not be NULL");
    if (dtype < 0 || dtype > 3) return fail(KL_ERR_INVALID_ARG, "bad dtype");
    if (!(cs >= 0) || !std::isfinite(cs)) return fail(KL_ERR_INVALID_ARG, "cs must be finite and >= 0");
    kl_status st = check_grid(grid, 1, nullptr);
    if (st) return st;
    const int es = esize_of(dtype);
    for (const void *p : {u, v, w, (const void *)nu})
        if ((uintptr_t)p % (uintptr_t)es) return fail(KL_ERR_INVALID_ARG, "field not aligned to its element size");
    if (u == nu || v == nu || w == nu) return fail(KL_ERR_INVALID_ARG, "nu must not alias u, v or w");
    Profile *prof = nullptr;
    st = get_profile(ctx, *grid, &prof);
    if (st) return st;
    // delta_k^2 per level, f64 then f32, one table per z grid, dx and dy (cs
    // enters as a kernel argument, so a new cs creates no table): the first
    // call on a grid allocates its table and uploads it synchronously
    std::vector<double> dzi, dzhi;
    zprofile_host(grid->nz, grid->g, grid->zbc, grid->zh, grid->dz, &dzi, &dzhi);
    std::vector<double> c64((size_t)grid->nz);
    for (int k = 0; k < grid->nz; ++k) {
        const double d = std::cbrt(grid->dx * grid->dy / dzi[(size_t)(k + grid->g)]);
        c64[(size_t)k] = d * d;
    }
    std::string key = "smag:" + std::to_string(fnv1a(c64.data(), c64.size() * sizeof(double)));
    auto it = ctx->tables.find(key);
    if (it == ctx->tables.end()) {
        size_t nb = c64.size() * (sizeof(double) + sizeof(float));
        std::vector<char> h(nb);
        memcpy(h.data(), c64.data(), c64.size() * sizeof(double));
        for (size_t k = 0; k < c64.size(); ++k) {
            float f = (float)c64[k];
            memcpy(h.data() + c64.size() * sizeof(double) + k * sizeof(float), &f, sizeof f);
        }
        void *d = nullptr;
        if (cudaMalloc(&d, nb) != cudaSuccess) return fail(KL_ERR_OOM, "cudaMalloc(smagorinsky table)");
        if (cudaMemcpy(d, h.data(), nb, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(d);
            return fail(KL_ERR_CUDA, "smagorinsky table upload");
        }
        it = ctx->tables.emplace(key, std::make_pair(d, nb)).first;
    }
    const double *cc64 = (const double *)it->second.first;
    const float *cc32 = (const float *)(cc64 + grid->nz);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = smag_launch(dtype, *grid, u, v, w, nu, prof->d64, prof->d32, prof->n, cc64, cc32,
                                cs * cs, s);
    if (e != cudaSuccess) return cuda_fail(e, "smagorinsky launch");
    ctx->launches++;
    if (fill_ghosts) {
        e = fill_ghosts_launch(es, *grid, nullptr, nullptr, nullptr, nu, s, true);
        if (e != cudaSuccess) return cuda_fail(e, "nu ghost fill");
        ctx->launches++;
    }
    return KL_OK;
}

kl_status kl_set_wait_limit(kl_ctx *ctx, int64_t cycles)
{
    if (!ctx || cycles < 0) return fail(KL_ERR_INVALID_ARG, "ctx is NULL or cycles < 0");
    ctx->wait_cycles = cycles ? (long long)cycles : kDefaultWaitCycles;
    return KL_OK;
}

kl_status kl_check(kl_ctx *ctx, void *stream)
{
    if (!ctx) return fail(KL_ERR_INVALID_ARG, "ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int word = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&word, ctx->d_err, sizeof word, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "kl_check: status read");
    if (!word) return KL_OK;
    e = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "kl_check: status reset");
    return fail(KL_ERR_TIMEOUT, "a device wait for a TMA plane gave up (status " +
                                    std::to_string(word) + "); the outputs of that launch are incomplete");
}

kl_status kl_stats(kl_ctx *ctx, char *buf, size_t n)
{
    if (!ctx || !buf || !n) return fail(KL_ERR_INVALID_ARG, "bad arguments");
    std::string rules;
    for (auto &p : ctx->selection_rule)
        rules += (rules.empty() ? "" : ",") + std::string("\"") + p.first + "\":" +
                 std::to_string(p.second);
    int m = snprintf(buf, n,
                     "{\"device\":\"%s\",\"cc\":\"%d.%d\",\"sms\":%d,\"launches\":%lld,"
                     "\"cache_hits\":%lld,\"cache_misses\":%lld,\"modules\":%zu,"
                     "\"stage_ms\":{\"wisdom\":%.3f,\"nvrtc\":%.3f,\"module_load\":%.3f,"
                     "\"launch\":%.3f},\"last_config\":\"%s\",\"last_batch\":\"%s\",\"rules\":{%s},\"note\":\"%s\","
                     "\"tables\":%zu,\"graphs\":%zu,\"graph_replays\":%lld,"
                     "\"disk_cache\":{\"on\":%s,\"hits\":%lld,\"writes\":%lld,\"read_ms\":%.3f}}",
                     ctx->name.c_str(), ctx->cc_major, ctx->cc_minor, ctx->nsm, ctx->launches,
                     ctx->cache_hits, ctx->cache_misses, ctx->kernels.size(), ctx->t_wisdom_ms,
                     ctx->t_nvrtc_ms, ctx->t_load_ms, ctx->t_launch_ms, ctx->last_config.c_str(),
                     ctx->last_batch.c_str(), rules.c_str(), ctx->last_rule_text.c_str(), ctx->tables.size(),
                     ctx->graphs.size(), ctx->graph_replays, ctx->cache_dir.empty() ? "false" : "true",
                     ctx->disk_hits, ctx->disk_writes, ctx->t_disk_ms);
    if (m < 0 || (size_t)m >= n) return fail(KL_ERR_INVALID_ARG, "stats buffer too small");
    return KL_OK;
}

// ---- host-only helpers

kl_status kl_config_normalize(const kl_op *op, const char *config, char *buf, size_t n)
{
    kl_status st = check_op(op);
    if (st) return st;
    if (!config || !buf) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    Config c;
    std::string err;
    if (!config_parse(config, &c, &err) || !config_check(*op, c, &err))
        return fail(KL_ERR_INVALID_ARG, err);
    std::string s = config_string(c);
    if (s.size() + 1 > n) return fail(KL_ERR_INVALID_ARG, "buffer too small");
    memcpy(buf, s.c_str(), s.size() + 1);
    return KL_OK;
}

kl_status kl_space_size(const kl_op *op, int32_t family, int64_t *count)
{
    kl_status st = check_op(op);
    if (st) return st;
    if (!count || family < 0 || family > 2) return fail(KL_ERR_INVALID_ARG, "bad family");
    *count = space_size(family);
    return KL_OK;
}

kl_status kl_space_config(const kl_op *op, int32_t family, int64_t idx, char *buf, size_t n)
{
    kl_status st = check_op(op);
    if (st) return st;
    Config c;
    if (!buf || !space_config(family, idx, &c)) return fail(KL_ERR_INVALID_ARG, "bad index");
    std::string s = config_string(c);
    if (s.size() + 1 > n) return fail(KL_ERR_INVALID_ARG, "buffer too small");
    memcpy(buf, s.c_str(), s.size() + 1);
    std::string err;
    if (!config_check(*op, c, &err)) return fail(KL_ERR_INVALID_ARG, err);
    return KL_OK;
}

kl_status kl_compile_only(const kl_op *op, const char *config, int32_t zbc, int32_t zuni,
                          char *log, size_t n)
{
    kl_status st = check_op(op);
    if (st) return st;
    Config c;
    std::string err, text = config ? config : "";
    bool batch = text.rfind("batch+", 0) == 0;     // "batch+<config>": the batched variant
    if (batch) text = text.substr(6);
    if (!config || !config_parse(text, &c, &err) || !config_check(*op, c, &err))
        return fail(KL_ERR_INVALID_ARG, "configuration: " + err);
    Compiled out;
    st = nvrtc_compile(compile_defines(*op, c, zbc, zuni) + (batch ? " -DKL_BATCH=1" : ""), true,
                       &out);
    if (log && n) {
        std::string s = st ? g_last_error : out.log;
        size_t m = std::min(n - 1, s.size());
        memcpy(log, s.data(), m);
        log[m] = '\0';
    }
    return st;
}

kl_status kl_set_cache_dir(kl_ctx *ctx, const char *dir)
{
    if (!ctx) return fail(KL_ERR_INVALID_ARG, "NULL context");
    if (!dir || !*dir) {
        ctx->cache_dir.clear();
        return KL_OK;
    }
    struct stat sb;
    if (stat(dir, &sb) != 0 || !S_ISDIR(sb.st_mode))
        return fail(KL_ERR_IO, std::string("cache directory does not exist: ") + dir);
    ctx->cache_dir = dir;
    return KL_OK;
}

kl_status kl_cache_prepare(const char *dir, const kl_op *op, const char *config, int32_t zbc,
                           int32_t zuni, int32_t *hit)
{
    kl_status st = check_op(op);
    if (st) return st;
    if (!dir || !*dir || !config || !hit) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    struct stat sb;
    if (stat(dir, &sb) != 0 || !S_ISDIR(sb.st_mode))
        return fail(KL_ERR_IO, std::string("cache directory does not exist: ") + dir);
    Config c;
    std::string err, text = config;
    bool batch = text.rfind("batch+", 0) == 0;
    if (batch) text = text.substr(6);
    if (!config_parse(text, &c, &err) || !config_check(*op, c, &err))
        return fail(KL_ERR_INVALID_ARG, "configuration: " + err);
    std::string key = compile_defines(*op, c, zbc, zuni) + (batch ? " -DKL_BATCH=1" : "");
    Compiled out;
    if (cache_read(dir, stencil_identity(key), &out)) {
        *hit = 1;
        return KL_OK;
    }
    *hit = 0;
    st = nvrtc_compile(key, false, &out);
    if (st) return st;
    if (!cache_write(dir, stencil_identity(key), out))
        return fail(KL_ERR_IO, std::string("cannot write into ") + dir);
    return KL_OK;
}

kl_status kl_wisdom_select(const char *path, const char *device, int32_t cc_major,
                           int32_t cc_minor, int32_t zbc, int32_t nx, int32_t ny, int32_t nz,
                           char *cfg, size_t n, int32_t *rule)
{
    if (!path || !device || !cfg || !n || !rule) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    std::vector<WisdomRecord> recs;
    std::string err, text = "default";
    int r = 5;
    kl_status st = KL_OK;
    if (wisdom_read(path, &recs, &err)) {
        r = wisdom_select(recs, device, cc_major, cc_minor, zbc, nx, ny, nz, &text);
    } else {
        // missing or unreadable file: the default (rule 5); report why
        set_error(err);
        st = KL_OK;
    }
    if (text.size() + 1 > n) return fail(KL_ERR_INVALID_ARG, "buffer too small");
    memcpy(cfg, text.c_str(), text.size() + 1);
    *rule = r;
    return st;
}

kl_status kl_wisdom_select_points(const char *path, const char *device, int32_t cc_major,
                                  int32_t cc_minor, int32_t zbc, int64_t points, char *cfg,
                                  size_t n, int32_t *rule)
{
    if (!path || !device || !cfg || !n || !rule) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    std::vector<WisdomRecord> recs;
    std::string err, text = "default";
    int r = 5;
    if (wisdom_read(path, &recs, &err))
        r = wisdom_select_points(recs, device, cc_major, cc_minor, zbc, (double)points, &text);
    else
        set_error(err);
    if (text.size() + 1 > n) return fail(KL_ERR_INVALID_ARG, "buffer too small");
    memcpy(cfg, text.c_str(), text.size() + 1);
    *rule = r;
    return KL_OK;
}

kl_status kl_wisdom_append(const char *path, const char *device, int32_t cc_major,
                           int32_t cc_minor, int32_t zbc, int32_t nx, int32_t ny, int32_t nz,
                           const char *config, double time_us, const char *extra)
{
    if (!path || !device || !config) return fail(KL_ERR_INVALID_ARG, "NULL argument");
    WisdomRecord r;
    r.device = device;
    r.cc_major = cc_major;
    r.cc_minor = cc_minor;
    r.zbc = zbc;
    r.nx = nx;
    r.ny = ny;
    r.nz = nz;
    r.config = config;
    r.time_us = time_us;
    if (extra && *extra) {
        std::stringstream ss(extra);
        std::string tok;
        while (ss >> tok) {
            size_t eq = tok.find('=');
            if (eq == std::string::npos) return fail(KL_ERR_INVALID_ARG, "extra needs key=value");
            r.extra[tok.substr(0, eq)] = tok.substr(eq + 1);
        }
    }
    std::string err;
    if (!wisdom_append(path, r, &err)) return fail(KL_ERR_IO, err);
    return KL_OK;
}

}  // extern "C"
