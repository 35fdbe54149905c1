// kl_internal.h -- declarations shared by the translation units of libkl.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "kl.h"

namespace kl {

// ------------------------------------------------------------ status
kl_status fail(kl_status code, const std::string &msg);   // records message, returns code
kl_status cuda_fail(cudaError_t e, const char *what);
kl_status cu_fail(CUresult r, const char *what);
void set_error(const std::string &msg);

// -------------------------------------------------------- configuration
// One point of the tuning space.  family 0 "direct": the parameters of
// Table 2.  family 1 "zmarch": z-marching CTAs with TMA-staged planes.
struct Config {
    int family = 0;
    // direct (Table 2 defaults)
    int bx = 256, by = 1, bz = 1;
    int tx = 1, ty = 1, tz = 1;
    int ux = 0, uy = 0, uz = 0;
    int cx = 0, cy = 0, cz = 0;
    int perm = 0;
    int minb = 1;
    // zmarch
    int mbx = 32, mby = 4;     // threads along x, y
    int mpx = 2, mpy = 1;      // points per thread along x (consecutive), y (block-strided)
    int kc = 32;               // z levels per CTA
    int ns = 8;                // plane ring slots (>= 7 + prefetch)
    int mminb = 1;             // min blocks per SM
    int yx = 0;                // zpack: exchange y faces between warps (shared memory)
    int pk = 1;                // zpack: packed f32x2 arithmetic (f32 compute)
    int cs = 0;                // zpack: one warp group per tendency component (3 x w warps)
    int pe = 0;                // zpack: persistent CTAs over (tile, level) ranges
};

// default deadline of one device wait, SM clock cycles (about a second)
constexpr long long kDefaultWaitCycles = 1ll << 31;

// storage type of the tendencies ut, vt, wt
inline int out_dtype(const kl_op &op) { return op.out_f32 ? (int)KL_F32 : op.dtype; }

// TMA descriptors per launch: u, v, w, nu with the plane box, then u, v, w
// with the 32-byte x-wrap strip box (zpack)
constexpr int KL_NMAPS = 7;

// threads of a z-march block along y (zpack with cs=1: three warp groups)
inline int zmarch_block_y(const Config &c) { return c.mby * (c.family == 2 && c.cs ? 3 : 1); }

std::string config_string(const Config &c);
bool config_parse(const std::string &s, Config *c, std::string *err);
// constraints of the space for an op (threads per block, shared memory,
// ghost width, ...).  smem_limit 0 = use the sm_103a per-block maximum.
bool config_check(const kl_op &op, const Config &c, std::string *err);
int64_t space_size(int family);

// Bayesian-optimisation surrogate (kl_bayes.cpp): fit a GP to n observations
// (X: n x d row-major features, y: values to minimise), add np pending points
// as kriging believers, and return the index of the candidate (C: m x d) of
// largest expected improvement (margin xi), or -1 with *err set.  ls <= 0
// selects the length scale by marginal likelihood (written to *ls_used).
int bo_suggest(int n, int d, const double *X, const double *y, int np, const double *P, int m,
               const double *C, double xi, double ls, double noise, double *ls_used,
               std::vector<double> *ei, std::string *err);
bool space_config(int family, int64_t idx, Config *c);

// tile / plane geometry of a zmarch configuration (mirrors the KL_* macros of
// the kernel source) and its dynamic shared memory in bytes
struct ZGeom {
    int al, txs, tys, lpad, pitch, rows, halo, nf;
    size_t box_bytes, plane_bytes;
};
ZGeom zmarch_geometry(const kl_op &op, const Config &c);
size_t zmarch_smem_bytes(const kl_op &op, const Config &c);
int halo_of(const kl_op &op);           // in-plane stencil reach (3 for adv5, else 1)
int esize_of(int dtype);

// ------------------------------------------------------------- wisdom
struct WisdomRecord {
    std::string device;
    int cc_major = 0, cc_minor = 0;
    int zbc = 0;
    int nx = 0, ny = 0, nz = 0;
    std::string config;
    double time_us = 0;
    std::map<std::string, std::string> extra;
};
bool wisdom_read(const std::string &path, std::vector<WisdomRecord> *out, std::string *err);
// returns rule 1..5 and the chosen configuration string
int wisdom_select(const std::vector<WisdomRecord> &recs, const std::string &device, int ccM,
                  int ccm, int zbc, int nx, int ny, int nz, std::string *config);
// rules 2..5 by the nearest point count (batched launches)
int wisdom_select_points(const std::vector<WisdomRecord> &recs, const std::string &device, int ccM,
                         int ccm, int zbc, double points, std::string *config);
std::string wisdom_file_name(const kl_op &op);
bool wisdom_append(const std::string &path, const WisdomRecord &r, std::string *err);

// ------------------------------------------------------------ compile
struct Compiled {
    std::vector<char> cubin;
    std::string log;
    std::string symbol;      // lowered name of the kernel function (user definitions)
};
// on-disk cubin cache (kl_api.cpp): identity of a variant from its source
// hash and compile options; read/write one variant's file in dir
uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull);
std::string cache_identity(uint64_t source_hash, const std::string &options);
bool cache_read(const std::string &dir, const std::string &ident, Compiled *out);
bool cache_write(const std::string &dir, const std::string &ident, const Compiled &c);
std::string compile_defines(const kl_op &op, const Config &c, int zbc, int zuni);
kl_status nvrtc_compile(const std::string &defines, bool verbose, Compiled *out);

// ------------------------------------------------------------ driver API
struct Driver {
    CUresult (*ModuleLoadData)(CUmodule *, const void *) = nullptr;
    CUresult (*ModuleUnload)(CUmodule) = nullptr;
    CUresult (*ModuleGetFunction)(CUfunction *, CUmodule, const char *) = nullptr;
    CUresult (*LaunchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned,
                             unsigned, unsigned, CUstream, void **, void **) = nullptr;
    CUresult (*FuncSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*OccupancyMaxActiveBlocksPerMultiprocessor)(int *, CUfunction, int, size_t) = nullptr;
    CUresult (*FuncGetAttribute)(int *, CUfunction_attribute, CUfunction) = nullptr;
    CUresult (*TensorMapEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                     const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                     const cuuint32_t *, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion,
                                     CUtensorMapFloatOOBfill) = nullptr;
};
kl_status driver_load(Driver *d);

// -------------------------------------------------------- kernel args
// Mirror of struct kl_args in kl_stencil.cuh (all members 8-byte aligned).
struct KArgs {
    const void *u, *v, *w, *nu;
    void *ut, *vt, *wt;
    const void *dzi, *dzhi;
    int *err;
    long long sj, sk;
    long long nx, ny, nz;
    long long nbx, nby, nbz;
    long long kchunk;
    long long tile_x0, tile_y0, tile_z0;
    double cd[8];
    float cf[8];
    long long wait_cycles;
    long long flags;            // bit 0: x, y ghosts supplied by the caller (grid.xybc)
};

struct Kernel {
    CUmodule mod = nullptr;
    CUfunction fn = nullptr;
    Config cfg;
    size_t smem = 0;
    int nregs = 0;
    int local_bytes = 0;
};

// a compiled user-defined kernel in a context (kl_def.cpp)
struct DefKernel {
    CUmodule mod = nullptr;
    CUfunction fn = nullptr;
    int smem_attr = 0;          // dynamic shared memory the function is opted in to
};
void def_kernels_unload(kl_ctx *ctx);

struct Profile {
    double *d64 = nullptr;   // dzi | dzhi, each nz + 2g, f64
    float *d32 = nullptr;    // same in f32
    int n = 0;
};

// validated geometry of one launch
struct Geom {
    int64_t x0, y0, z0;      // tensor coordinates of interior (0,0,0)
};
kl_status check_grid(const kl_grid *g, int need_g, Geom *geo);
void zprofile_host(int nz, int g, int zbc, const double *zh, double dz_uniform,
                   std::vector<double> *dzi, std::vector<double> *dzhi);

}  // namespace kl

struct kl_ctx {
    int device = 0;
    int cc_major = 0, cc_minor = 0;
    int nsm = 0;
    std::string name;
    std::string wisdom_dir;
    kl::Driver drv;
    std::map<std::string, kl::Kernel> kernels;        // compile key -> module
    std::map<std::string, std::string> selection;     // problem key -> config
    std::map<std::string, int> selection_rule;
    std::map<std::string, kl::Profile> profiles;      // z-grid key -> device profiles
    int *d_err = nullptr;
    double *d_scratch = nullptr;
    size_t scratch_doubles = 0;
    double *h_out = nullptr;                          // pinned, diag results
    // tile tables of batched launches, keyed by the batch signature
    std::map<std::string, std::pair<void *, size_t>> tables;
    std::map<std::string, CUtensorMap> tmaps;         // TMA descriptors per buffer/box
    // streams that run the configuration classes of one batched call side by
    // side (forked from and joined back into the caller's stream)
    std::vector<cudaStream_t> aux_streams;
    std::vector<cudaEvent_t> aux_events;              // [0] fork, [1 + i] join of stream i
    // one executable CUDA graph per batch (op, grids, fields) seen before
    std::map<std::string, cudaGraphExec_t> graphs;
    long long wait_cycles = kl::kDefaultWaitCycles;   // limit of one device wait
    cudaStream_t cap_stream = nullptr;                // where batch graphs are recorded
    long long graph_replays = 0;
    // statistics
    long long launches = 0, cache_hits = 0, cache_misses = 0;
    double t_wisdom_ms = 0, t_nvrtc_ms = 0, t_load_ms = 0, t_launch_ms = 0;
    double last_first_launch_ms = 0;
    // on-disk cubin cache (empty: off; $KL_CACHE_DIR at creation)
    std::string cache_dir;
    long long disk_hits = 0, disk_writes = 0;
    // user-defined kernels, keyed by their cache identity
    std::map<std::string, kl::DefKernel> def_kernels;
    double t_disk_ms = 0;
    std::string last_config, last_rule_text;
    std::string last_batch;    // classes of the last batch planned: "config xN; ..."
};

namespace kl {
// launch one tendency kernel with a resolved configuration (shared by
// kl_launch, kl_launch_with_config and the tuner)
kl_status launch_config(kl_ctx *ctx, const kl_op &op, const Config &cfg, const kl_grid &g,
                        const kl_fields &f, cudaStream_t s);
// cache key and NVRTC defines of a kernel in a context: compile_defines,
// plus KL_WAITPOLL=1 when the context's wait limit differs from the default
std::string kernel_key(const kl_ctx *ctx, const kl_op &op, const Config &cfg, int zbc, int zuni);
kl_status get_kernel(kl_ctx *ctx, const kl_op &op, const Config &cfg, int zbc, int zuni,
                     Kernel **out, bool batch = false);
// kernel arguments and TMA descriptors of one launch (validated)
kl_status make_kargs(kl_ctx *ctx, const kl_op &op, const Config &cfg, const kl_grid &g,
                     const kl_fields &f, KArgs *a, CUtensorMap maps[KL_NMAPS]);
kl_status select_config(kl_ctx *ctx, const kl_op &op, const kl_grid &g, Config *cfg);
// the configuration of a batch of `points` interior points of boundary zbc
kl_status select_batch_config(kl_ctx *ctx, const kl_op &op, int zbc, long long points, Config *cfg);
kl_status check_op(const kl_op *op);
kl_status check_fields(const kl_op &op, const kl_fields *f);
kl_status get_profile(kl_ctx *ctx, const kl_grid &g, Profile **out);
// can configuration cfg run on this grid's memory layout and pointers?
bool config_fits(const kl_op &op, const Config &cfg, const kl_grid &g, const kl_fields *f,
                 std::string *why);
// device kernels of kl_device.cu
// x_ghosts false: leave the x ghosts of interior rows of interior levels as
// they are (fill the y rows and z planes only)
void halo_strip_shape(const kl_grid &g, int axis, int *w, int *h);
cudaError_t halo_launch(int esize, const kl_grid &g, int axis, int side, int nf, void *const *fields,
                        void *buf, bool unpack, cudaStream_t s);
cudaError_t fill_ghosts_launch(int esize, const kl_grid &g, void *u, void *v, void *w,
                               void *nu, cudaStream_t s, bool x_ghosts = true);
cudaError_t diag_launch(int dtype, const kl_grid &g, int level, const void *t,
                        const double *ref, const double *wz, double *scratch, int nblocks,
                        double *dout, cudaStream_t s);
int diag_blocks(int nsm);
cudaError_t dot_launch(int dtype, const kl_grid &g, const void *x, const void *y,
                       const double *wz, double *scratch, int nblocks, double *dout,
                       cudaStream_t s);
cudaError_t compare_launch(int dtype, const kl_grid &g, const void *a, const void *b,
                           unsigned long long *dout, int nsm, cudaStream_t s);
// Smagorinsky viscosity at the interior cell centres (profile arrays of get_profile)
cudaError_t smag_launch(int dtype, const kl_grid &g, const void *u, const void *v, const void *w,
                        void *nu, const double *d64, const float *d32, int nprof,
                        const double *cc64, const float *cc32, double cs2, cudaStream_t s);
// load a compiled cubin into the context's cache under its compile key
kl_status load_compiled(kl_ctx *ctx, const kl_op &op, const Config &cfg, const std::string &key,
                        const Compiled &c, Kernel **out);
}  // namespace kl
