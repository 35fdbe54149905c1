// kl_device.cu -- ghost fill and FP64 diagnostic reductions (nvcc, sm_103a).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "kl_internal.h"

namespace {

// ------------------------------------------------------------ ghost fill
//
// Ghost points form three disjoint groups: the 2g full z planes (x and y
// ghosts included), the 2g y rows of every interior level (x ghosts
// included), and the 2g x points of every interior row.  Each ghost maps
// straight to an interior source point, axis by axis, so one launch fills
// faces, edges and corners with no ordering between them (no source is ever a
// ghost).  The copy moves raw bits; the odd (w) mirror flips the sign bit,
// which negates exactly in every format.
//
// The first blocks take the rows of the first two groups, one padded row per
// warp: the row's source row is found once, and the lanes sweep x with
// FILL_RU cells each in flight (all loads before any store).  The last blocks
// take the x ghosts of interior rows through one linear cell index, FILL_U
// cells per thread.

constexpr int FILL_T = 256, FILL_W = FILL_T / 32, FILL_RU = 9, FILL_U = 4;

struct FillArgs {
    char *f[4];              // u, v, w, nu at interior (0,0,0); NULL: not filled
    long long sj, sk;
    int nx, ny, nz, zbc;
    int rows_z, rows_y;      // rows of the z-plane group (2g x padded ny), y-row group (2g x nz)
    int nb_rows;             // blocks of the row groups
    unsigned n_x;            // cells of the x group (0: not filled)
    int xyhalo;              // 1: x, y ghosts belong to the caller (z planes only,
                             // each ghost from its own column, no x / y wrap)
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// source levels of ghost level k: even mirror / periodic (ske), odd mirror (sko)
__device__ __forceinline__ void fill_levels(const FillArgs &a, int k, int &ske, int &sko,
                                            bool &wzero, bool &wneg)
{
    if (a.zbc == 0) {
        ske = sko = wrapi(k, a.nz);
        wzero = wneg = false;
    } else {
        ske = k < 0 ? -1 - k : (k >= a.nz ? 2 * a.nz - 1 - k : k);
        sko = k < 0 ? -k : (k > a.nz ? 2 * a.nz - k : k);
        wzero = k == a.nz;
        wneg = k < 0 || k > a.nz;
    }
}

template <typename B>
__device__ __forceinline__ B fill_w(B v, bool wzero, bool wneg)
{
    const B sign_bit = (B)1 << (sizeof(B) * 8 - 1);
    return wzero ? (B)0 : (wneg ? (B)(v ^ sign_bit) : v);
}

// one padded row (x in [-G, nx + G)) at (j, k), by one warp
template <typename B, int G>
__device__ __forceinline__ void fill_row(const FillArgs &a, int j, int k, int lane)
{
    int ske, sko;
    bool wzero, wneg;
    fill_levels(a, k, ske, sko, wzero, wneg);
    const long long sj = a.xyhalo ? j : wrapi(j, a.ny);
    const long long dst0 = j * a.sj + k * a.sk;
    const long long src0 = sj * a.sj + ske * a.sk, srcw0 = sj * a.sj + sko * a.sk;
    for (int i0 = -G; i0 < a.nx + G; i0 += 32 * FILL_RU) {
        B val[FILL_RU][4];
#pragma unroll
        for (int c = 0; c < FILL_RU; ++c) {
            const int i = i0 + lane + 32 * c;
            if (i >= a.nx + G) continue;
            const int si = a.xyhalo ? i : wrapi(i, a.nx);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (!a.f[f]) continue;
                const B *p = (const B *)a.f[f];
                if (f != 2) val[c][f] = p[src0 + si];
                else if (!wzero) val[c][f] = p[srcw0 + si];
            }
        }
#pragma unroll
        for (int c = 0; c < FILL_RU; ++c) {
            const int i = i0 + lane + 32 * c;
            if (i >= a.nx + G) continue;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (!a.f[f]) continue;
                ((B *)a.f[f])[dst0 + i] = f != 2 ? val[c][f] : fill_w<B>(val[c][f], wzero, wneg);
            }
        }
    }
}

template <typename B, int G>
__global__ void __launch_bounds__(FILL_T) fill_kernel(FillArgs a)
{
    if ((int)blockIdx.x < a.nb_rows) {
        // row groups: warp -> row task r
        const int r = (int)blockIdx.x * FILL_W + (int)(threadIdx.x >> 5);
        if (r >= a.rows_z + a.rows_y) return;
        int j, k;
        if (r < a.rows_z) {                // z planes: 2G planes of ny + 2G rows
            const int py = a.ny + 2 * G, p = r / py;
            j = r - p * py - G;
            k = p < G ? p - G : a.nz + (p - G);
        } else {                           // y rows: 2G rows of every interior level
            const int t = r - a.rows_z, kk = t / (2 * G), qq = t - kk * (2 * G);
            j = qq < G ? qq - G : a.ny + (qq - G);
            k = kk;
        }
        fill_row<B, G>(a, j, k, (int)(threadIdx.x & 31));
        return;
    }
    // x ghosts of interior rows: 2G points x ny rows x nz levels, linear
    const unsigned base = ((unsigned)blockIdx.x - a.nb_rows) * (unsigned)(FILL_T * FILL_U) + threadIdx.x;
    long long dst[FILL_U], src[FILL_U], srcw[FILL_U];
    bool live[FILL_U];
#pragma unroll
    for (int c = 0; c < FILL_U; ++c) {
        const unsigned q = base + c * FILL_T;
        live[c] = q < a.n_x;
        const unsigned rr = q / (2 * G), qq = q - rr * (2 * G), kk = live[c] ? rr / (unsigned)a.ny : 0;
        const int i = qq < (unsigned)G ? (int)qq - G : a.nx + ((int)qq - G);
        const int j = (int)(rr - kk * (unsigned)a.ny), k = (int)kk;
        const int si = wrapi(i, a.nx);
        dst[c] = i + j * a.sj + k * a.sk;
        src[c] = si + j * a.sj + k * a.sk;       // interior row: only x wraps
        srcw[c] = src[c];
    }
    B val[FILL_U][4];
#pragma unroll
    for (int c = 0; c < FILL_U; ++c) {
        if (!live[c]) continue;
#pragma unroll
        for (int f = 0; f < 4; ++f)
            if (a.f[f]) val[c][f] = ((const B *)a.f[f])[f == 2 ? srcw[c] : src[c]];
    }
#pragma unroll
    for (int c = 0; c < FILL_U; ++c) {
        if (!live[c]) continue;
#pragma unroll
        for (int f = 0; f < 4; ++f)
            if (a.f[f]) ((B *)a.f[f])[dst[c]] = val[c][f];
    }
}

template <typename B>
static cudaError_t fill_dispatch(int g, unsigned grid, const FillArgs &a, cudaStream_t s)
{
    switch (g) {
    case 1: fill_kernel<B, 1><<<grid, FILL_T, 0, s>>>(a); break;
    case 2: fill_kernel<B, 2><<<grid, FILL_T, 0, s>>>(a); break;
    case 3: fill_kernel<B, 3><<<grid, FILL_T, 0, s>>>(a); break;
    case 4: fill_kernel<B, 4><<<grid, FILL_T, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ----------------------------------------------------- halo strips
//
// Pack / unpack of one halo strip of an x-y decomposed block (kl_halo_pack,
// kl_halo_unpack): a box of W columns x H rows x nz levels at (x0, y0, 0) of
// up to 4 fields <-> a contiguous buffer [field][k][row][column].  One thread
// per element, raw bits (B = the storage word), x fastest so that the y
// strips (whole padded rows) move in coalesced runs.

struct HaloArgs {
    char *f[4];              // fields at interior (0,0,0)
    char *buf;
    long long sj, sk;
    int x0, y0, w, h, nz, nf;
    int unpack;              // 0: fields -> buf, 1: buf -> fields
};

template <typename B>
__global__ void __launch_bounds__(256) halo_kernel(HaloArgs a)
{
    const long long n = (long long)a.w * a.h * a.nz * a.nf;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        long long r = q;
        const int i = (int)(r % a.w);
        r /= a.w;
        const int j = (int)(r % a.h);
        r /= a.h;
        const int k = (int)(r % a.nz);
        const int f = (int)(r / a.nz);
        B *p = (B *)a.f[f] + ((long long)(a.x0 + i) + (long long)(a.y0 + j) * a.sj + (long long)k * a.sk);
        B *b = (B *)a.buf + q;
        if (a.unpack)
            *p = *b;
        else
            *b = *p;
    }
}

}  // namespace

namespace kl {

// W x H of the strip of `axis`
void halo_strip_shape(const kl_grid &g, int axis, int *w, int *h)
{
    *w = axis == 0 ? g.g : g.nx + 2 * g.g;
    *h = axis == 0 ? g.ny : g.g;
}

cudaError_t halo_launch(int esize, const kl_grid &g, int axis, int side, int nf, void *const *fields,
                        void *buf, bool unpack, cudaStream_t s)
{
    HaloArgs a;
    size_t off = (size_t)g.origin * esize;
    for (int f = 0; f < 4; ++f) a.f[f] = f < nf ? (char *)fields[f] + off : nullptr;
    a.buf = (char *)buf;
    a.sj = g.sj;
    a.sk = g.sk;
    halo_strip_shape(g, axis, &a.w, &a.h);
    a.nz = g.nz;
    a.nf = nf;
    a.unpack = unpack ? 1 : 0;
    if (axis == 0) {
        a.x0 = unpack ? (side ? g.nx : -g.g) : (side ? g.nx - g.g : 0);
        a.y0 = 0;
    } else {
        a.x0 = -g.g;
        a.y0 = unpack ? (side ? g.ny : -g.g) : (side ? g.ny - g.g : 0);
    }
    const long long n = (long long)a.w * a.h * a.nz * nf;
    if (n == 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 1LL << 20);
    if (esize == 8)
        halo_kernel<unsigned long long><<<(unsigned)blocks, 256, 0, s>>>(a);
    else if (esize == 4)
        halo_kernel<unsigned int><<<(unsigned)blocks, 256, 0, s>>>(a);
    else
        halo_kernel<unsigned short><<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace kl

namespace {

// ---------------------------------------------------------- diagnostics

struct DiagArgs {
    const void *t;
    const double *ref;
    const double *wz;        // weight per level k (dz_k or dzh_k)
    long long sj, sk;
    int nx, ny, nz;
    long long n;
    double *partial;         // nblocks x 6
};

template <typename T> __device__ __forceinline__ double to_d(T x) { return (double)x; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
template <> __device__ __forceinline__ double to_d<__half>(__half x) { return (double)__half2float(x); }

__device__ __forceinline__ void reduce6(double v[6], double *out)
{
    // 0, 2: max; others: sum
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 6; ++c) {
            double x = __shfl_xor_sync(0xffffffffu, v[c], o);
            v[c] = (c == 0 || c == 2) ? fmax(v[c], x) : v[c] + x;
        }
    __shared__ double sh[32][6];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int c = 0; c < 6; ++c) sh[warp][c] = v[c];
    __syncthreads();
    if (warp == 0) {
        for (int c = 0; c < 6; ++c) v[c] = lane < nw ? sh[lane][c] : ((c == 0 || c == 2) ? 0.0 : 0.0);
        for (int o = 16; o > 0; o >>= 1)
            for (int c = 0; c < 6; ++c) {
                double x = __shfl_xor_sync(0xffffffffu, v[c], o);
                v[c] = (c == 0 || c == 2) ? fmax(v[c], x) : v[c] + x;
            }
        if (lane == 0)
            for (int c = 0; c < 6; ++c) out[c] = v[c];
    }
}

// float-float accumulator: hi + lo carries the sum of FP32 values with about
// 48 significant bits; every addition is Knuth's error-free TwoSum, products
// of two floats enter exactly through their FMA residual
struct kl_ff { float hi, lo; };

__device__ __forceinline__ void ff_add(kl_ff &acc, float x)
{
    const float s = acc.hi + x;
    const float bp = s - acc.hi;
    const float err = (acc.hi - (s - bp)) + (x - bp);
    acc.hi = s;
    acc.lo += err;
}

__device__ __forceinline__ void ff_add_square(kl_ff &acc, float x)
{
    const float p = x * x;
    const float pe = fmaf(x, x, -p);          // x*x = p + pe exactly
    ff_add(acc, p);
    acc.lo += pe;
}

__device__ __forceinline__ double ff_value(const kl_ff &acc) { return (double)acc.hi + (double)acc.lo; }

// Each warp takes a contiguous block of interior rows (j, k) (consecutive
// rows of a level lie next to each other in memory), lanes along x, every
// load coalesced.  Without a reference (the common case: t in f32 or 16-bit
// storage) the per-element work stays in FP32: the maximum is exact in FP32
// and the sums run in float-float; a lane folds its float-float partials into
// FP64 once per level it touches (the dz-weighted sum takes that level's sum
// times w_k).  GB300 runs FP64 at a small fraction of its FP32 rate, which is
// what this keeps off the per-element path.  With f64 storage every element
// is reduced in FP64.  With an FP64 reference and f32 or 16-bit storage the
// difference e = t - ref and the two sums of squares stay FP64 (one
// subtraction, two FMAs per element: their relative accuracy is the FP64
// one), the two maxima are taken as integer maxima of the magnitudes' bit
// patterns (IEEE order of non-negative doubles, no FP64 work) and the sum of
// t runs in float-float as above.
template <typename T, bool REF>
__global__ void __launch_bounds__(256) diag_kernel(DiagArgs a)
{
    double v[6] = {0, 0, 0, 0, 0, 0};
    const T *t = (const T *)a.t;
    const int lane = (int)(threadIdx.x & 31);
    const long long rows = (long long)a.ny * a.nz;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long per = (rows + nw - 1) / nw;
    const long long rb = wid * per, re = rb + per < rows ? rb + per : rows;
    if (rb < re) {
        int k = (int)(rb / a.ny), j = (int)(rb - (long long)k * a.ny);
        float tmax = 0.0f;
        kl_ff s1 = {0.0f, 0.0f}, s2 = {0.0f, 0.0f};      // this level's sum and squares
        double rs = 0.0;                                 // this level's sum (FP64 path)
        unsigned long long emax = 0, rmax = 0;           // |e|, |ref| maxima as bit patterns
        constexpr unsigned long long kMag = 0x7fffffffffffffffull;
        for (long long r = rb; r < re; ++r) {
            const long long o0 = j * a.sj + (long long)k * a.sk;
            if (REF && sizeof(T) != 8) {
                for (int i0 = lane; i0 < a.nx; i0 += 32 * 4) {
                    float x[4];
                    double rv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const bool in = i0 + 32 * u < a.nx;
                        x[u] = in ? (float)to_d(t[o0 + i0 + 32 * u]) : 0.0f;
                        rv[u] = in ? a.ref[o0 + i0 + 32 * u] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const double e = (double)x[u] - rv[u];
                        const unsigned long long eb = (unsigned long long)__double_as_longlong(e) & kMag;
                        const unsigned long long rbits =
                            (unsigned long long)__double_as_longlong(rv[u]) & kMag;
                        emax = eb > emax ? eb : emax;
                        rmax = rbits > rmax ? rbits : rmax;
                        v[1] = fma(e, e, v[1]);
                        v[3] = fma(rv[u], rv[u], v[3]);
                        ff_add(s1, x[u]);
                    }
                }
            } else if (REF || sizeof(T) == 8) {
#pragma unroll 4
                for (int i = lane; i < a.nx; i += 32) {
                    const double tv = to_d(t[o0 + i]);
                    const double rv = REF ? a.ref[o0 + i] : 0.0;
                    const double e = tv - rv;
                    v[0] = fmax(v[0], fabs(e));
                    v[1] = fma(e, e, v[1]);
                    if (REF) {
                        v[2] = fmax(v[2], fabs(rv));
                        v[3] = fma(rv, rv, v[3]);
                    }
                    rs += tv;
                }
            } else {
                // eight loads per lane in flight before the arithmetic
                for (int i0 = lane; i0 < a.nx; i0 += 32 * 8) {
                    float x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        x[u] = i0 + 32 * u < a.nx ? (float)to_d(t[o0 + i0 + 32 * u]) : 0.0f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        tmax = fmaxf(tmax, fabsf(x[u]));
                        ff_add(s1, x[u]);
                        ff_add_square(s2, x[u]);
                    }
                }
            }
            // next row; at the end of a level (or of the block) fold the level's sum
            if (++j == a.ny || r + 1 == re) {
                const double ls = sizeof(T) == 8 ? rs : ff_value(s1);
                v[4] += ls;
                v[5] = fma(ls, a.wz[k], v[5]);
                if (!(REF || sizeof(T) == 8)) v[1] += ff_value(s2);
                rs = 0.0;
                s1.hi = s1.lo = 0.0f;
                s2.hi = s2.lo = 0.0f;
                if (j == a.ny) {
                    j = 0;
                    ++k;
                }
            }
        }
        if (!(REF || sizeof(T) == 8)) v[0] = fmax(v[0], (double)tmax);
        if (REF && sizeof(T) != 8) {
            v[0] = fmax(v[0], __longlong_as_double((long long)emax));
            v[2] = fmax(v[2], __longlong_as_double((long long)rmax));
        }
    }
    reduce6(v, a.partial + 6 * (size_t)blockIdx.x);
}

// inner product sum a*b over the interior, weighted per level by wz[k] (wz
// NULL: weight 1), in the layout of diag_kernel: f32 and 16-bit products are
// exact FP32 pairs (p + FMA residual) summed in float-float and folded into
// FP64 once per level; f64 products are summed in FP64.  The block's partial
// goes to record slot 4 (the other slots are zero), which diag_final sums.
template <typename T>
__global__ void __launch_bounds__(256) dot_kernel(DiagArgs a, const void *bptr)
{
    double acc = 0.0;
    const T *x = (const T *)a.t, *y = (const T *)bptr;
    const int lane = (int)(threadIdx.x & 31);
    const long long rows = (long long)a.ny * a.nz;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long per = (rows + nw - 1) / nw;
    const long long rb = wid * per, re = rb + per < rows ? rb + per : rows;
    if (rb < re) {
        int k = (int)(rb / a.ny), j = (int)(rb - (long long)k * a.ny);
        kl_ff s = {0.0f, 0.0f};
        double ds = 0.0;
        for (long long r = rb; r < re; ++r) {
            const long long o0 = j * a.sj + (long long)k * a.sk;
            if (sizeof(T) == 8) {
                for (int i = lane; i < a.nx; i += 32) ds = fma(to_d(x[o0 + i]), to_d(y[o0 + i]), ds);
            } else {
                for (int i0 = lane; i0 < a.nx; i0 += 32 * 4) {
                    float xa[4], ya[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const bool in = i0 + 32 * u < a.nx;
                        xa[u] = in ? (float)to_d(x[o0 + i0 + 32 * u]) : 0.0f;
                        ya[u] = in ? (float)to_d(y[o0 + i0 + 32 * u]) : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float p = xa[u] * ya[u];
                        const float pe = fmaf(xa[u], ya[u], -p);   // xa*ya = p + pe exactly
                        ff_add(s, p);
                        s.lo += pe;
                    }
                }
            }
            if (++j == a.ny || r + 1 == re) {
                const double ls = sizeof(T) == 8 ? ds : ff_value(s);
                acc = a.wz ? fma(ls, a.wz[k], acc) : acc + ls;
                ds = 0.0;
                s.hi = s.lo = 0.0f;
                if (j == a.ny) {
                    j = 0;
                    ++k;
                }
            }
        }
    }
    double v[6] = {0, 0, 0, 0, acc, 0};
    reduce6(v, a.partial + 6 * (size_t)blockIdx.x);
}

__global__ void __launch_bounds__(256) diag_final(const double *partial, int nb, long long n, double *out)
{
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double *p = partial + 6 * (size_t)b;
        v[0] = fmax(v[0], p[0]);
        v[1] += p[1];
        v[2] = fmax(v[2], p[2]);
        v[3] += p[3];
        v[4] += p[4];
        v[5] += p[5];
    }
    __shared__ double res[6];
    reduce6(v, res);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = res[0];
        out[1] = n ? sqrt(res[1] / (double)n) : 0.0;
        out[2] = res[2];
        out[3] = n ? sqrt(res[3] / (double)n) : 0.0;
        out[4] = res[4];
        out[5] = res[5];
    }
}

}  // namespace

namespace kl {

cudaError_t fill_ghosts_launch(int esize, const kl_grid &g, void *u, void *v, void *w, void *nu,
                               cudaStream_t s, bool x_ghosts)
{
    if (g.g < 1 || g.g > 4) return cudaErrorInvalidValue;
    FillArgs a;
    size_t off = (size_t)g.origin * esize;
    a.f[0] = u ? (char *)u + off : nullptr;     // any field may be absent
    a.f[1] = v ? (char *)v + off : nullptr;
    a.f[2] = w ? (char *)w + off : nullptr;
    a.f[3] = nu ? (char *)nu + off : nullptr;
    a.sj = g.sj;
    a.sk = g.sk;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.zbc = g.zbc;
    // a decomposed block (xybc = 1): the z planes only; its x and y ghosts
    // hold the neighbours' halo
    a.xyhalo = g.xybc ? 1 : 0;
    long long rows_z = 2LL * g.g * (g.ny + 2LL * g.g), rows_y = g.xybc ? 0 : 2LL * g.g * g.nz;
    long long n_x = x_ghosts && !g.xybc ? 2LL * g.g * g.ny * g.nz : 0;
    long long nb_rows = (rows_z + rows_y + FILL_W - 1) / FILL_W;
    long long nb_x = (n_x + FILL_T * FILL_U - 1) / (FILL_T * FILL_U);
    // 32-bit row and cell indices (the last x block's cells included)
    if (rows_z + rows_y > 0x7fffffffLL || n_x + FILL_T * FILL_U > 0xffffffffLL ||
        nb_rows + nb_x > 0x7fffffffLL)
        return cudaErrorInvalidValue;
    a.rows_z = (int)rows_z;
    a.rows_y = (int)rows_y;
    a.nb_rows = (int)nb_rows;
    a.n_x = (unsigned)n_x;
    unsigned grid = (unsigned)(nb_rows + nb_x);
    if (esize == 8) return fill_dispatch<unsigned long long>(g.g, grid, a, s);
    if (esize == 4) return fill_dispatch<unsigned int>(g.g, grid, a, s);
    return fill_dispatch<unsigned short>(g.g, grid, a, s);
}

int diag_blocks(int nsm) { return nsm * 8; }

// At most nmax blocks of 256 threads, and no more than fit on the device at
// once: the reductions give each warp a fixed share of the rows, so a partial
// second wave would double the time of the blocks it holds.
template <typename K>
static int one_wave(K kernel, int nmax)
{
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, 0) != cudaSuccess)
        return nmax;
    return std::max(1, std::min(nmax, per * nsm));
}

cudaError_t diag_launch(int dtype, const kl_grid &g, int level, const void *t, const double *ref,
                        const double *wz, double *scratch, int nblocks, double *dout,
                        cudaStream_t s)
{
    (void)level;
    int es = esize_of(dtype);
    DiagArgs a;
    a.t = (const char *)t + (size_t)g.origin * es;
    a.ref = ref ? ref + g.origin : nullptr;
    a.wz = wz;
    a.sj = g.sj;
    a.sk = g.sk;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.n = (long long)g.nx * g.ny * g.nz;
    a.partial = scratch;
    auto go = [&](auto kernel) {
        nblocks = one_wave(kernel, nblocks);
        kernel<<<nblocks, 256, 0, s>>>(a);
    };
    switch (dtype * 2 + (ref ? 1 : 0)) {
    case 2 * KL_F64: go(diag_kernel<double, false>); break;
    case 2 * KL_F64 + 1: go(diag_kernel<double, true>); break;
    case 2 * KL_F32: go(diag_kernel<float, false>); break;
    case 2 * KL_F32 + 1: go(diag_kernel<float, true>); break;
    case 2 * KL_BF16: go(diag_kernel<__nv_bfloat16, false>); break;
    case 2 * KL_BF16 + 1: go(diag_kernel<__nv_bfloat16, true>); break;
    case 2 * KL_F16: go(diag_kernel<__half, false>); break;
    default: go(diag_kernel<__half, true>); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, 256, 0, s>>>(scratch, nblocks, a.n, dout);
    return cudaGetLastError();
}

cudaError_t dot_launch(int dtype, const kl_grid &g, const void *x, const void *y,
                       const double *wz, double *scratch, int nblocks, double *dout,
                       cudaStream_t s)
{
    int es = esize_of(dtype);
    DiagArgs a;
    a.t = (const char *)x + (size_t)g.origin * es;
    a.ref = nullptr;
    a.wz = wz;
    a.sj = g.sj;
    a.sk = g.sk;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.n = (long long)g.nx * g.ny * g.nz;
    a.partial = scratch;
    const void *yb = (const char *)y + (size_t)g.origin * es;
    auto go = [&](auto kernel) {
        nblocks = one_wave(kernel, nblocks);
        kernel<<<nblocks, 256, 0, s>>>(a, yb);
    };
    switch (dtype) {
    case KL_F64: go(dot_kernel<double>); break;
    case KL_F32: go(dot_kernel<float>); break;
    case KL_BF16: go(dot_kernel<__nv_bfloat16>); break;
    default: go(dot_kernel<__half>); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, 256, 0, s>>>(scratch, nblocks, a.n, dout);
    return cudaGetLastError();
}

}  // namespace kl

// ==================================================== allocation-free diag
//
// kl_diag_noalloc is for callers that may not allocate GPU memory while they
// run: applications that reserve their whole device-memory budget up front
// and own the allocator, or time loops that cannot afford the implicit device
// synchronisation and possible failure of cudaMalloc between steps.  Its
// scratch (one partial record of 6 doubles per block of KL_NOALLOC_PTS
// points, plus the 6 results) is this file-scope array, which every GPU that
// loads the library keeps until the process exits.  Every call overwrites the
// records it uses before reading them, so nothing has to start at zero; the
// array is shared by all calls, so calls that overlap on the GPU (different
// streams, or host threads) race and must be serialised by the caller.

#define KL_NOALLOC_PTS 8192                    // interior points per block
#define KL_NOALLOC_MAX_BLOCKS 8192             // => at most 2^26 interior points
static __device__ __align__(256) double kl_noalloc_scratch[KL_NOALLOC_MAX_BLOCKS * 6 + 8];

namespace {

// As diag_kernel, but block b reduces the fixed point range
// [b * KL_NOALLOC_PTS, (b + 1) * KL_NOALLOC_PTS), so the number of partial
// records depends on the grid only.  wz may be NULL (weights 1).
template <typename T>
__global__ void __launch_bounds__(256) diag_kernel_fixed(DiagArgs a)
{
    double v[6] = {0, 0, 0, 0, 0, 0};
    const T *t = (const T *)a.t;
    long long q0 = (long long)blockIdx.x * KL_NOALLOC_PTS;
    long long q1 = q0 + KL_NOALLOC_PTS < a.n ? q0 + KL_NOALLOC_PTS : a.n;
    for (long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int i = (int)(q % a.nx);
        long long r = q / a.nx;
        int j = (int)(r % a.ny);
        int k = (int)(r / a.ny);
        long long o = i + j * a.sj + k * a.sk;
        double tv = to_d(t[o]);
        double rv = a.ref ? a.ref[o] : 0.0;
        double e = tv - rv;
        v[0] = fmax(v[0], fabs(e));
        v[1] += e * e;
        v[2] = fmax(v[2], fabs(rv));
        v[3] += rv * rv;
        v[4] += tv;
        v[5] += tv * (a.wz ? a.wz[k] : 1.0);
    }
    reduce6(v, a.partial + 6 * (size_t)blockIdx.x);
}

// device address of kl_noalloc_scratch per device, looked up once per device
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[256] = {nullptr};

}  // namespace

extern "C" kl_status kl_diag_noalloc(int32_t dtype, const kl_grid *grid, const void *t,
                                     const double *ref, const double *wz, double out[6],
                                     void *stream)
{
    using namespace kl;
    if (!t || !out) return fail(KL_ERR_INVALID_ARG, "kl_diag_noalloc: t and out must not be NULL");
    if (dtype < 0 || dtype > 3) return fail(KL_ERR_INVALID_ARG, "kl_diag_noalloc: dtype must be 0..3");
    kl_status st = check_grid(grid, 1, nullptr);
    if (st) return st;
    long long n = (long long)grid->nx * grid->ny * grid->nz;
    long long nb = (n + KL_NOALLOC_PTS - 1) / KL_NOALLOC_PTS;
    if (nb > KL_NOALLOC_MAX_BLOCKS)
        return fail(KL_ERR_INVALID_ARG,
                    "kl_diag_noalloc: grid has " + std::to_string(n) +
                        " interior points; the static scratch holds at most " +
                        std::to_string((long long)KL_NOALLOC_MAX_BLOCKS * KL_NOALLOC_PTS) +
                        " (use kl_diag)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "kl_diag_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 256) return fail(KL_ERR_UNSUPPORTED, "kl_diag_noalloc: device index >= 256");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // set-up, once per device, with that device current: the host-side
            // name of the array is not a device address, so ask the runtime
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, kl_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "kl_diag_noalloc: cudaGetSymbolAddress");
            g_noalloc_ptr[dev] = (double *)p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    int es = esize_of(dtype);
    DiagArgs a;
    a.t = (const char *)t + (size_t)grid->origin * es;
    a.ref = ref ? ref + grid->origin : nullptr;
    a.wz = wz;
    a.sj = grid->sj;
    a.sk = grid->sk;
    a.nx = grid->nx;
    a.ny = grid->ny;
    a.nz = grid->nz;
    a.n = n;
    a.partial = scratch;
    cudaStream_t s = (cudaStream_t)stream;
    switch (dtype) {
    case KL_F64: diag_kernel_fixed<double><<<(unsigned)nb, 256, 0, s>>>(a); break;
    case KL_F32: diag_kernel_fixed<float><<<(unsigned)nb, 256, 0, s>>>(a); break;
    case KL_BF16: diag_kernel_fixed<__nv_bfloat16><<<(unsigned)nb, 256, 0, s>>>(a); break;
    default: diag_kernel_fixed<__half><<<(unsigned)nb, 256, 0, s>>>(a); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kl_diag_noalloc: launch");
    double *res = scratch + (size_t)KL_NOALLOC_MAX_BLOCKS * 6;
    diag_final<<<1, 256, 0, s>>>(scratch, (int)nb, n, res);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kl_diag_noalloc: launch");
    e = cudaMemcpyAsync(out, res, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "kl_diag_noalloc: readback");
    return KL_OK;
}

// ============================================ output comparison (tuner)
//
// max |a - b| and max |b| over the interior of two fields of the same type,
// accumulated as non-negative doubles by an integer atomicMax on their bits
// (the order of non-negative IEEE doubles is the order of their bit patterns).

namespace {

template <typename T>
__global__ void __launch_bounds__(256) compare_kernel(const T *a, const T *b, long long sj,
                                                      long long sk, int nx, int ny, long long n,
                                                      unsigned long long *out)
{
    double e = 0.0, m = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        int i = (int)(q % nx);
        long long r = q / nx;
        int j = (int)(r % ny);
        int k = (int)(r / ny);
        long long o = i + j * sj + k * sk;
        double x = to_d(a[o]), y = to_d(b[o]);
        double d = fabs(x - y);
        if (!(d <= 1e300)) d = 1e300;   // NaN or inf: worst possible
        e = fmax(e, d);
        m = fmax(m, fabs(y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(e));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(m));
    }
}

}  // namespace

namespace kl {

cudaError_t compare_launch(int dtype, const kl_grid &g, const void *a, const void *b,
                           unsigned long long *dout, int nsm, cudaStream_t s)
{
    int es = esize_of(dtype);
    const char *pa = (const char *)a + (size_t)g.origin * es;
    const char *pb = (const char *)b + (size_t)g.origin * es;
    long long n = (long long)g.nx * g.ny * g.nz;
    cudaError_t e = cudaMemsetAsync(dout, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int nb = nsm * 4;
    switch (dtype) {
    case KL_F64: compare_kernel<double><<<nb, 256, 0, s>>>((const double *)pa, (const double *)pb, g.sj, g.sk, g.nx, g.ny, n, dout); break;
    case KL_F32: compare_kernel<float><<<nb, 256, 0, s>>>((const float *)pa, (const float *)pb, g.sj, g.sk, g.nx, g.ny, n, dout); break;
    case KL_BF16: compare_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>((const __nv_bfloat16 *)pa, (const __nv_bfloat16 *)pb, g.sj, g.sk, g.nx, g.ny, n, dout); break;
    default: compare_kernel<__half><<<nb, 256, 0, s>>>((const __half *)pa, (const __half *)pb, g.sj, g.sk, g.nx, g.ny, n, dout); break;
    }
    return cudaGetLastError();
}

}  // namespace kl

namespace {

// ------------------------------------------------- Smagorinsky viscosity
//
// nu = (cs delta_k)^2 sqrt(2 S_ij S_ij) at the interior cell centres,
// delta_k = (dx dy dz_k)^(1/3), the factor per level from a table; the normal strains at the centre, each shear
// strain squared on the four edges around the cell and averaged, so
//   2 S_ij S_ij = 2 (Sxx^2 + Syy^2 + Szz^2) + sum over the 12 edges of e^2,
// e = (d_i u_j + d_j u_i)/2 on the edge.  One thread per (i, j) column marches
// up SMAG_KC levels: the values of its own column at the current level and the
// two vertical-edge strains above it carry into the next level, so each level
// reads 17 values (9 at k+1, 8 neighbours at k), all coalesced along x.
// HBM-bound: u, v, w read once from memory, nu written once.

constexpr int SMAG_BX = 32, SMAG_BY = 8;

struct SmagArgs {
    const void *u, *v, *w;   // at interior (0,0,0)
    void *nu;
    const double *dzi64, *dzhi64;          // index k + g
    const float *dzi32, *dzhi32;
    const double *cc64;                    // delta_k^2, index k
    const float *cc32;
    double cs2;                            // cs^2
    long long sj, sk;
    int nx, ny, nz, g, kc;
    double dxi, dyi;
};

template <typename T> __device__ __forceinline__ float ldf(const T *p) { return (float)*p; }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ float ldf<__half>(const __half *p) { return __half2float(*p); }
template <typename T> __device__ __forceinline__ void stf(T *p, float x) { *p = (T)x; }
template <> __device__ __forceinline__ void stf<__nv_bfloat16>(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ void stf<__half>(__half *p, float x) { *p = __float2half_rn(x); }

// compute type C: double for f64 storage, float otherwise
template <typename T, typename C>
__device__ __forceinline__ C ldc(const T *p) { return (C)ldf<T>(p); }
template <>
__device__ __forceinline__ double ldc<double, double>(const double *p) { return *p; }

template <typename T, typename C>
__global__ void __launch_bounds__(SMAG_BX * SMAG_BY) smag_kernel(SmagArgs a)
{
    const int i = blockIdx.x * SMAG_BX + threadIdx.x;
    const int j = blockIdx.y * SMAG_BY + threadIdx.y;
    const int k0 = blockIdx.z * a.kc;
    if (i >= a.nx || j >= a.ny || k0 >= a.nz) return;
    const int k1 = min(k0 + a.kc, a.nz);
    const T *u = (const T *)a.u, *v = (const T *)a.v, *w = (const T *)a.w;
    T *nu = (T *)a.nu;
    const long long sj = a.sj, sk = a.sk;
    const C dxi = (C)a.dxi, dyi = (C)a.dyi, half = (C)0.5;
    auto dzi = [&](int k) { return sizeof(C) == 8 ? (C)a.dzi64[k + a.g] : (C)a.dzi32[k + a.g]; };
    auto dzhi = [&](int k) { return sizeof(C) == 8 ? (C)a.dzhi64[k + a.g] : (C)a.dzhi32[k + a.g]; };

    long long o = i + j * sj + (long long)k0 * sk;
    // own column at level k0, and the vertical-edge strains on the face below
    C u0 = ldc<T, C>(u + o), u1 = ldc<T, C>(u + o + 1);
    C v0 = ldc<T, C>(v + o), v1 = ldc<T, C>(v + o + sj);
    C w0 = ldc<T, C>(w + o);
    C exz0, exz1, eyz0, eyz1;
    {
        const C zi = dzhi(k0);
        exz0 = half * ((u0 - ldc<T, C>(u + o - sk)) * zi + (w0 - ldc<T, C>(w + o - 1)) * dxi);
        exz1 = half * ((u1 - ldc<T, C>(u + o + 1 - sk)) * zi + (ldc<T, C>(w + o + 1) - w0) * dxi);
        eyz0 = half * ((v0 - ldc<T, C>(v + o - sk)) * zi + (w0 - ldc<T, C>(w + o - sj)) * dyi);
        eyz1 = half * ((v1 - ldc<T, C>(v + o + sj - sk)) * zi + (ldc<T, C>(w + o + sj) - w0) * dyi);
    }
    for (int k = k0; k < k1; ++k, o += sk) {
        const long long p = o + sk;
        // level k + 1: own column and the faces above
        const C u0n = ldc<T, C>(u + p), u1n = ldc<T, C>(u + p + 1);
        const C v0n = ldc<T, C>(v + p), v1n = ldc<T, C>(v + p + sj);
        const C w0n = ldc<T, C>(w + p);
        const C wxm = ldc<T, C>(w + p - 1), wxp = ldc<T, C>(w + p + 1);
        const C wym = ldc<T, C>(w + p - sj), wyp = ldc<T, C>(w + p + sj);
        // level k: the neighbours of the horizontal edges
        const C uym0 = ldc<T, C>(u + o - sj), uym1 = ldc<T, C>(u + o + 1 - sj);
        const C uyp0 = ldc<T, C>(u + o + sj), uyp1 = ldc<T, C>(u + o + 1 + sj);
        const C vxm0 = ldc<T, C>(v + o - 1), vxp0 = ldc<T, C>(v + o + 1);
        const C vxm1 = ldc<T, C>(v + o - 1 + sj), vxp1 = ldc<T, C>(v + o + 1 + sj);

        const C zi = dzhi(k + 1);
        const C exz0n = half * ((u0n - u0) * zi + (w0n - wxm) * dxi);
        const C exz1n = half * ((u1n - u1) * zi + (wxp - w0n) * dxi);
        const C eyz0n = half * ((v0n - v0) * zi + (w0n - wym) * dyi);
        const C eyz1n = half * ((v1n - v1) * zi + (wyp - w0n) * dyi);
        const C sxx = (u1 - u0) * dxi, syy = (v1 - v0) * dyi, szz = (w0n - w0) * dzi(k);
        const C e00 = half * ((u0 - uym0) * dyi + (v0 - vxm0) * dxi);
        const C e10 = half * ((u1 - uym1) * dyi + (vxp0 - v0) * dxi);
        const C e01 = half * ((uyp0 - u0) * dyi + (v1 - vxm1) * dxi);
        const C e11 = half * ((uyp1 - u1) * dyi + (vxp1 - v1) * dxi);
        C s2 = (C)2 * (sxx * sxx + syy * syy + szz * szz);
        s2 += e00 * e00 + e10 * e10 + e01 * e01 + e11 * e11;
        s2 += exz0 * exz0 + exz1 * exz1 + exz0n * exz0n + exz1n * exz1n;
        s2 += eyz0 * eyz0 + eyz1 * eyz1 + eyz0n * eyz0n + eyz1n * eyz1n;
        const C cc = (C)a.cs2 * (sizeof(C) == 8 ? (C)a.cc64[k] : (C)a.cc32[k]);
        const C val = cc * sqrt(s2);
        if (sizeof(C) == 8) ((double *)nu)[o] = (double)val;
        else stf<T>(nu + o, (float)val);
        u0 = u0n; u1 = u1n; v0 = v0n; v1 = v1n; w0 = w0n;
        exz0 = exz0n; exz1 = exz1n; eyz0 = eyz0n; eyz1 = eyz1n;
    }
}

// Four x-points per thread (i = 4t .. 4t+3) with 4-wide loads: used when nx,
// the interior origin and both strides are multiples of 4 elements and the
// fields are aligned to 4 elements, so every 4-wide access starts inside
// the interior row and the single-element x neighbours (i - 1, i + 4) are
// interior points or the first ghost.  The vertical-edge strains of the five
// x-edges and of the two y-edges of the four points carry from one level to
// the next, and each horizontal edge strain serves the two points beside it.

template <typename T, typename C> struct Quad;
template <> struct Quad<float, float> {
    static __device__ __forceinline__ void ld(const float *p, float o[4])
    {
        const float4 x = *(const float4 *)p;
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
    }
    static __device__ __forceinline__ void st(float *p, const float o[4])
    {
        *(float4 *)p = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <> struct Quad<double, double> {
    static __device__ __forceinline__ void ld(const double *p, double o[4])
    {
        const double2 a = ((const double2 *)p)[0], b = ((const double2 *)p)[1];
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
    static __device__ __forceinline__ void st(double *p, const double o[4])
    {
        ((double2 *)p)[0] = make_double2(o[0], o[1]);
        ((double2 *)p)[1] = make_double2(o[2], o[3]);
    }
};
template <> struct Quad<__nv_bfloat16, float> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, float o[4])
    {
        const __nv_bfloat162 *q = (const __nv_bfloat162 *)p;
        const float2 a = __bfloat1622float2(q[0]), b = __bfloat1622float2(q[1]);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, const float o[4])
    {
        __nv_bfloat162 *q = (__nv_bfloat162 *)p;
        q[0] = __float22bfloat162_rn(make_float2(o[0], o[1]));
        q[1] = __float22bfloat162_rn(make_float2(o[2], o[3]));
    }
};
template <> struct Quad<__half, float> {
    static __device__ __forceinline__ void ld(const __half *p, float o[4])
    {
        const __half2 *q = (const __half2 *)p;
        const float2 a = __half22float2(q[0]), b = __half22float2(q[1]);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
    static __device__ __forceinline__ void st(__half *p, const float o[4])
    {
        __half2 *q = (__half2 *)p;
        q[0] = __float22half2_rn(make_float2(o[0], o[1]));
        q[1] = __float22half2_rn(make_float2(o[2], o[3]));
    }
};

// One level of the R-row, four-point layout: the values a thread reads at
// level k + 1 (its rows, v on their faces, w in the rows below and above
// them) and at level k (u in rows j - 1 and j + R, v at x = i - 1 and i + 4).
template <typename C, int R>
struct SmagLevel {
    C Un[R][5], Vn[R + 1][4], Wn[R][4], Wm[4], Wp[4], wl[R], wr[R];
    C Ujm[5], Ujp[5], vm[R + 1], vp[R + 1];
};

// The strains of one level and nu at the thread's 4 x R points, from the
// carried level-k values (U, V, W and the vertical-edge strains below) and
// the level's reads L; EXZn, EYZn are the vertical-edge strains above.
template <typename C, int R>
__device__ __forceinline__ void smag_level_math(const SmagLevel<C, R> &L, const C (&U)[R][5],
                                                const C (&V)[R + 1][4], const C (&W)[R][4],
                                                const C (&EXZ)[R][5], const C (&EYZ)[R + 1][4],
                                                C zi, C dzik, C dxi, C dyi, C cc,
                                                C (&EXZn)[R][5], C (&EYZn)[R + 1][4], C (&out)[R][4])
{
    const C half = (C)0.5;
    C E[R + 1][5];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            const C whi = e == 4 ? L.wr[r] : L.Wn[r][e], wlo = e == 0 ? L.wl[r] : L.Wn[r][e - 1];
            EXZn[r][e] = half * ((L.Un[r][e] - U[r][e]) * zi + (whi - wlo) * dxi);
        }
#pragma unroll
    for (int y = 0; y <= R; ++y) {
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            const C uhi = y == R ? L.Ujp[e] : U[y][e], ulo = y == 0 ? L.Ujm[e] : U[y - 1][e];
            const C vr = e == 4 ? L.vp[y] : V[y][e], vl = e == 0 ? L.vm[y] : V[y][e - 1];
            E[y][e] = half * ((uhi - ulo) * dyi + (vr - vl) * dxi);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const C whi = y == R ? L.Wp[q] : L.Wn[y][q], wlo = y == 0 ? L.Wm[q] : L.Wn[y - 1][q];
            EYZn[y][q] = half * ((L.Vn[y][q] - V[y][q]) * zi + (whi - wlo) * dyi);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const C sxx = (U[r][q + 1] - U[r][q]) * dxi, syy = (V[r + 1][q] - V[r][q]) * dyi;
            const C szz = (L.Wn[r][q] - W[r][q]) * dzik;
            C s2 = (C)2 * (sxx * sxx + syy * syy + szz * szz);
            s2 += E[r][q] * E[r][q] + E[r][q + 1] * E[r][q + 1] + E[r + 1][q] * E[r + 1][q] +
                  E[r + 1][q + 1] * E[r + 1][q + 1];
            s2 += EXZ[r][q] * EXZ[r][q] + EXZ[r][q + 1] * EXZ[r][q + 1] + EXZn[r][q] * EXZn[r][q] +
                  EXZn[r][q + 1] * EXZn[r][q + 1];
            s2 += EYZ[r][q] * EYZ[r][q] + EYZ[r + 1][q] * EYZ[r + 1][q] + EYZn[r][q] * EYZn[r][q] +
                  EYZn[r + 1][q] * EYZn[r + 1][q];
            out[r][q] = cc * sqrt(s2);
        }
}

// Carry level k + 1 into the level-k state.
template <typename C, int R>
__device__ __forceinline__ void smag_carry(const SmagLevel<C, R> &L, const C (&EXZn)[R][5],
                                           const C (&EYZn)[R + 1][4], C (&U)[R][5], C (&V)[R + 1][4],
                                           C (&W)[R][4], C (&EXZ)[R][5], C (&EYZ)[R + 1][4])
{
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            U[r][e] = L.Un[r][e];
            EXZ[r][e] = EXZn[r][e];
        }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) W[r][q] = L.Wn[r][q];
#pragma unroll
    for (int y = 0; y <= R; ++y)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            V[y][q] = L.Vn[y][q];
            EYZ[y][q] = EYZn[y][q];
        }
}

// R consecutive rows per thread (j .. j+R-1): the R + 1 y-edges of those rows
// are formed once per level, so two rows share the strains of the edge
// between them and the loads of the rows next to it (25 loads per level for
// 8 points at R = 2 against 34 at R = 1).  Every point is formed with the
// same operations in the same order whatever R (the compiler may contract
// different products into FMAs in the two instances).
template <typename T, typename C, int R>
__global__ void __launch_bounds__(SMAG_BX * SMAG_BY, sizeof(C) == 8 ? 1 : (R == 1 ? 3 : 2))
smag_kernel4(SmagArgs a)
{
    using Q = Quad<T, C>;
    const int i = 4 * (blockIdx.x * SMAG_BX + threadIdx.x);
    const int j = R * (blockIdx.y * SMAG_BY + threadIdx.y);
    const int k0 = blockIdx.z * a.kc;
    if (i >= a.nx || j >= a.ny || k0 >= a.nz) return;
    const int k1 = min(k0 + a.kc, a.nz);
    const T *u = (const T *)a.u, *v = (const T *)a.v, *w = (const T *)a.w;
    T *nu = (T *)a.nu;
    const long long sj = a.sj, sk = a.sk;
    const C dxi = (C)a.dxi, dyi = (C)a.dyi, half = (C)0.5;
    auto dzi = [&](int k) { return sizeof(C) == 8 ? (C)a.dzi64[k + a.g] : (C)a.dzi32[k + a.g]; };
    auto dzhi = [&](int k) { return sizeof(C) == 8 ? (C)a.dzhi64[k + a.g] : (C)a.dzhi32[k + a.g]; };

    long long o = i + j * sj + (long long)k0 * sk;
    // level k0: u at x = i .. i+4 and w in rows j .. j+R-1, v on the y faces
    // of rows j .. j+R; then the edge strains on the face below (x-edges at
    // i .. i+4 of each row, y-edges at yh_j .. yh_{j+R})
    C U[R][5], V[R + 1][4], W[R][4], EXZ[R][5], EYZ[R + 1][4];
    {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Q::ld(u + o + r * sj, U[r]);
            U[r][4] = ldc<T, C>(u + o + r * sj + 4);
            Q::ld(w + o + r * sj, W[r]);
        }
#pragma unroll
        for (int e = 0; e <= R; ++e) Q::ld(v + o + e * sj, V[e]);
        const C zi = dzhi(k0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C Ub[5];
            Q::ld(u + o + r * sj - sk, Ub);
            Ub[4] = ldc<T, C>(u + o + r * sj + 4 - sk);
            const C wl = ldc<T, C>(w + o + r * sj - 1), wr = ldc<T, C>(w + o + r * sj + 4);
#pragma unroll
            for (int e = 0; e < 5; ++e) {
                const C whi = e == 4 ? wr : W[r][e], wlo = e == 0 ? wl : W[r][e - 1];
                EXZ[r][e] = half * ((U[r][e] - Ub[e]) * zi + (whi - wlo) * dxi);
            }
        }
        C Wm[4], Wp[4];
        Q::ld(w + o - sj, Wm);
        Q::ld(w + o + R * sj, Wp);
#pragma unroll
        for (int e = 0; e <= R; ++e) {
            C Vb[4];
            Q::ld(v + o + e * sj - sk, Vb);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const C whi = e == R ? Wp[q] : W[e][q], wlo = e == 0 ? Wm[q] : W[e - 1][q];
                EYZ[e][q] = half * ((V[e][q] - Vb[q]) * zi + (whi - wlo) * dyi);
            }
        }
    }
    for (int k = k0; k < k1; ++k, o += sk) {
        const long long p = o + sk;
        SmagLevel<C, R> L;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Q::ld(u + p + r * sj, L.Un[r]);
            L.Un[r][4] = ldc<T, C>(u + p + r * sj + 4);
            Q::ld(w + p + r * sj, L.Wn[r]);
            L.wl[r] = ldc<T, C>(w + p + r * sj - 1);
            L.wr[r] = ldc<T, C>(w + p + r * sj + 4);
        }
#pragma unroll
        for (int e = 0; e <= R; ++e) Q::ld(v + p + e * sj, L.Vn[e]);
        Q::ld(w + p - sj, L.Wm);
        Q::ld(w + p + R * sj, L.Wp);
        Q::ld(u + o - sj, L.Ujm);
        L.Ujm[4] = ldc<T, C>(u + o + 4 - sj);
        Q::ld(u + o + R * sj, L.Ujp);
        L.Ujp[4] = ldc<T, C>(u + o + 4 + R * sj);
#pragma unroll
        for (int e = 0; e <= R; ++e) {
            L.vm[e] = ldc<T, C>(v + o + e * sj - 1);
            L.vp[e] = ldc<T, C>(v + o + e * sj + 4);
        }
        const C cc = (C)a.cs2 * (sizeof(C) == 8 ? (C)a.cc64[k] : (C)a.cc32[k]);
        C EXZn[R][5], EYZn[R + 1][4], out[R][4];
        smag_level_math<C, R>(L, U, V, W, EXZ, EYZ, dzhi(k + 1), dzi(k), dxi, dyi, cc, EXZn, EYZn, out);
#pragma unroll
        for (int r = 0; r < R; ++r) Q::st(nu + o + r * sj, out[r]);
        smag_carry<C, R>(L, EXZn, EYZn, U, V, W, EXZ, EYZ);
    }
}

}  // namespace

namespace kl {

cudaError_t smag_launch(int dtype, const kl_grid &g, const void *u, const void *v, const void *w,
                        void *nu, const double *d64, const float *d32, int nprof,
                        const double *cc64, const float *cc32, double cs2, cudaStream_t s)
{
    const int es = esize_of(dtype);
    const size_t off = (size_t)g.origin * es;
    SmagArgs a;
    a.cs2 = cs2;
    a.u = (const char *)u + off;
    a.v = (const char *)v + off;
    a.w = (const char *)w + off;
    a.nu = (char *)nu + off;
    a.dzi64 = d64;
    a.dzhi64 = d64 + nprof;
    a.dzi32 = d32;
    a.dzhi32 = d32 + nprof;
    a.cc64 = cc64;
    a.cc32 = cc32;
    a.sj = g.sj;
    a.sk = g.sk;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.g = g.g;
    a.kc = 16;
    a.dxi = 1.0 / g.dx;
    a.dyi = 1.0 / g.dy;
    dim3 block(SMAG_BX, SMAG_BY);
    const uintptr_t al = 4 * (uintptr_t)es;
    const bool quad = g.nx % 4 == 0 && g.origin % 4 == 0 && g.sj % 4 == 0 && g.sk % 4 == 0 &&
                      (uintptr_t)u % al == 0 && (uintptr_t)v % al == 0 && (uintptr_t)w % al == 0 &&
                      (uintptr_t)nu % al == 0;
    if (quad) {
        // two rows per thread where ny is even (every thread's second row is
        // interior) and the compute type is f32; one otherwise
        const int R = g.ny % 2 == 0 && dtype != KL_F64 ? 2 : 1;
        dim3 grid((g.nx / 4 + SMAG_BX - 1) / SMAG_BX, (g.ny / R + SMAG_BY - 1) / SMAG_BY,
                  (g.nz + a.kc - 1) / a.kc);
        if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
        switch (dtype) {
        case KL_F64: smag_kernel4<double, double, 1><<<grid, block, 0, s>>>(a); break;
        case KL_F32:
            if (R == 2) {
                smag_kernel4<float, float, 2><<<grid, block, 0, s>>>(a);
            } else {
                smag_kernel4<float, float, 1><<<grid, block, 0, s>>>(a);
            }
            break;
        case KL_BF16:
            if (R == 2) smag_kernel4<__nv_bfloat16, float, 2><<<grid, block, 0, s>>>(a);
            else smag_kernel4<__nv_bfloat16, float, 1><<<grid, block, 0, s>>>(a);
            break;
        default:
            if (R == 2) smag_kernel4<__half, float, 2><<<grid, block, 0, s>>>(a);
            else smag_kernel4<__half, float, 1><<<grid, block, 0, s>>>(a);
            break;
        }
        return cudaGetLastError();
    }
    dim3 grid((g.nx + SMAG_BX - 1) / SMAG_BX, (g.ny + SMAG_BY - 1) / SMAG_BY, (g.nz + a.kc - 1) / a.kc);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    switch (dtype) {
    case KL_F64: smag_kernel<double, double><<<grid, block, 0, s>>>(a); break;
    case KL_F32: smag_kernel<float, float><<<grid, block, 0, s>>>(a); break;
    case KL_BF16: smag_kernel<__nv_bfloat16, float><<<grid, block, 0, s>>>(a); break;
    default: smag_kernel<__half, float><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace kl
