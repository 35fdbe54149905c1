// kl_stencil.cuh -- tendency kernels, compiled at run time by NVRTC for sm_103a.
//
// Every tunable parameter and every problem option arrives as a -D define, so
// each configuration is its own specialised cubin (Sec. 4.5: parameter values
// are compile-time constants of the runtime-compiled instance).
//
// Problem defines:
//   KL_DTYPE   0 f64, 1 f32, 2 bf16, 3 f16 (storage type; f64 computes in f64,
//              the others in f32)
//   KL_ADV     0 none, 2 centred 2nd order, 5 upwind-biased 5th order
//   KL_DIFF    0 none, 1 constant-nu Laplacian, 2 variable-nu stress divergence
//   KL_ZBC     0 periodic z, 1 free-slip walls (wt = 0 on the bottom wall face)
//   KL_ZUNI    1 uniform dz (scalars), 0 profiles dzi[k], dzhi[k]
//   KL_ACC     0 t = tendency, 1 t += tendency
// Family KL_FAMILY 0 ("direct", the tunable space of Table 2):
//   KL_BX KL_BY KL_BZ  thread-block shape
//   KL_TX KL_TY KL_TZ  points per thread along each axis (tile factors)
//   KL_UX KL_UY KL_UZ  fully unroll the tile loop of that axis
//   KL_CX KL_CY KL_CZ  1: a thread's points are consecutive, 0: block-strided
//   KL_PERM            unravel order of the 1D block index (0 XYZ 1 XZY 2 YXZ
//                      3 YZX 4 ZXY 5 ZYX, first letter fastest)
//   KL_MINB            minimum resident blocks per SM (__launch_bounds__)
// Family KL_FAMILY 1 ("zmarch"): see the second half of this file.
//
// Discretisation (staggered Arakawa-C grid; u at (xh_i, y_j, z_k), v at
// (x_i, yh_j, z_k), w at (x_i, y_j, zh_k), nu at centres):
//   flux-form advection -div(u_j u_i) with face fluxes F = U * a_face, U the
//   2-point mean of the carrying velocity, a_face the 2-point mean (2nd order)
//   or the upwind-biased 5th-order value U*I6 + |U|*D6 (Wicker-Skamarock);
//   nu * Laplacian or the stress divergence d_j[nu (d_j u_i + d_i u_j)] with
//   4-point edge averages of nu.  These are the MicroHH advec_u / diff_uvw
//   operators named in Sec. 5.2, generalised to all three components.

#ifndef KL_DTYPE
#error "KL_DTYPE must be defined"
#endif

typedef unsigned short kl_u16;

#if KL_DTYPE == 0
typedef double T;
typedef double C;
#elif KL_DTYPE == 1
typedef float T;
typedef float C;
#else
typedef kl_u16 T;
typedef float C;
#endif

// Kernel argument block; the host fills an identical struct (8-byte members).
struct kl_args {
    const T *u, *v, *w, *nu;      // pointers at interior point (0,0,0)
    T *ut, *vt, *wt;
    const C *dzi, *dzhi;          // profiles, index k = interior level (may be < 0)
    int *err;                     // device status word (0 = ok)
    long long sj, sk;             // element strides of y and z
    long long nx, ny, nz;
    long long nbx, nby, nbz;      // blocks per axis (direct family)
    long long kchunk;             // z levels per CTA (zmarch family)
    long long tile_x0, tile_y0, tile_z0;  // tensor coordinates of interior (0,0,0)
    // coefficients, precomputed on the host in both precisions so that an
    // f32 kernel does no f64 arithmetic: dxi, dyi, dzi0, dzhi0, nu, nu*dxi^2,
    // nu*dyi^2, unused
    double cd[8];
    float cf[8];
};

#if KL_DTYPE == 0
#define KL_CO(a, i) ((a).cd[i])
#else
#define KL_CO(a, i) ((a).cf[i])
#endif

// ---------------------------------------------------------------- storage

__device__ __forceinline__ C ld(const T *p)
{
#if KL_DTYPE == 2
    return __uint_as_float(((unsigned)__ldg(p)) << 16);
#elif KL_DTYPE == 3
    float f;
    kl_u16 h = __ldg(p);
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
    return f;
#else
    return __ldg(p);
#endif
}

__device__ __forceinline__ C lds(const T *p)   // plain (shared or generic) load
{
#if KL_DTYPE == 2
    return __uint_as_float(((unsigned)*p) << 16);
#elif KL_DTYPE == 3
    float f;
    kl_u16 h = *p;
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
    return f;
#else
    return *p;
#endif
}

__device__ __forceinline__ void st(T *p, C v)
{
#if KL_DTYPE == 2
    kl_u16 r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(v));
    *p = r;
#elif KL_DTYPE == 3
    kl_u16 r;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(r) : "f"(v));
    *p = r;
#else
    *p = v;
#endif
}

__device__ __forceinline__ void out(T *p, C v)
{
#if KL_ACC
    v += lds(p);
#endif
    st(p, v);
}

// ------------------------------------------------------------ face fluxes
//
// Us is twice the advecting velocity (sum of two neighbours); a0..a5 are the
// advected values around the face (face between a2 and a3).  The returned
// flux is scaled by KL_FS_INV; the caller multiplies by KL_FS.
//   5th order: 120 F = Us*(37(a2+a3) - 8(a1+a4) + (a0+a5))
//                     + |Us|*(10(a2-a3) - 5(a1-a4) + (a0-a5))
//   2nd order:   4 F = Us*(a2+a3)

__device__ __forceinline__ C flux5(C Us, C a0, C a1, C a2, C a3, C a4, C a5)
{
    C s1 = a2 + a3, s2 = a1 + a4, s3 = a0 + a5;
    C d1 = a2 - a3, d2 = a1 - a4, d3 = a0 - a5;
    C i6 = fma(C(37), s1, fma(C(-8), s2, s3));
    C d6 = fma(C(10), d1, fma(C(-5), d2, d3));
    return fma(Us, i6, fabs(Us) * d6);
}

__device__ __forceinline__ C flux2(C Us, C a2, C a3) { return Us * (a2 + a3); }

#if KL_ADV == 5
#define KL_FLUX(Us, a0, a1, a2, a3, a4, a5) flux5((Us), (a0), (a1), (a2), (a3), (a4), (a5))
#define KL_FS (C(1) / C(120))
#else
#define KL_FLUX(Us, a0, a1, a2, a3, a4, a5) flux2((Us), (a2), (a3))
#define KL_FS (C(0.25))
#endif

// ---------------------------------------------------- one-point tendency
//
// A is an accessor with template members U<di,dj,dk>(), V<>, W<>, N<> that
// return the field value at the given offset from the point.  zc carries the
// vertical metric of the level: dzi_k, dzhi_k, dzhi_{k+1}, dzi_{k-1}.

struct kl_zmetric { C dzi, dzhi, dzhi_up, dzi_dn; };

#define Uf(a, b, c) A.template U<(a), (b), (c)>()
#define Vf(a, b, c) A.template V<(a), (b), (c)>()
#define Wf(a, b, c) A.template W<(a), (b), (c)>()
#define Nf(a, b, c) A.template N<(a), (b), (c)>()

// u momentum
#define FUX(m) KL_FLUX(Uf(m, 0, 0) + Uf(m + 1, 0, 0), Uf(m - 2, 0, 0), Uf(m - 1, 0, 0), \
                       Uf(m, 0, 0), Uf(m + 1, 0, 0), Uf(m + 2, 0, 0), Uf(m + 3, 0, 0))
#define FUY(m) KL_FLUX(Vf(-1, m, 0) + Vf(0, m, 0), Uf(0, m - 3, 0), Uf(0, m - 2, 0), \
                       Uf(0, m - 1, 0), Uf(0, m, 0), Uf(0, m + 1, 0), Uf(0, m + 2, 0))
#define FUZ(m) KL_FLUX(Wf(-1, 0, m) + Wf(0, 0, m), Uf(0, 0, m - 3), Uf(0, 0, m - 2), \
                       Uf(0, 0, m - 1), Uf(0, 0, m), Uf(0, 0, m + 1), Uf(0, 0, m + 2))
// v momentum
#define FVX(m) KL_FLUX(Uf(m, -1, 0) + Uf(m, 0, 0), Vf(m - 3, 0, 0), Vf(m - 2, 0, 0), \
                       Vf(m - 1, 0, 0), Vf(m, 0, 0), Vf(m + 1, 0, 0), Vf(m + 2, 0, 0))
#define FVY(m) KL_FLUX(Vf(0, m, 0) + Vf(0, m + 1, 0), Vf(0, m - 2, 0), Vf(0, m - 1, 0), \
                       Vf(0, m, 0), Vf(0, m + 1, 0), Vf(0, m + 2, 0), Vf(0, m + 3, 0))
#define FVZ(m) KL_FLUX(Wf(0, -1, m) + Wf(0, 0, m), Vf(0, 0, m - 3), Vf(0, 0, m - 2), \
                       Vf(0, 0, m - 1), Vf(0, 0, m), Vf(0, 0, m + 1), Vf(0, 0, m + 2))
// w momentum
#define FWX(m) KL_FLUX(Uf(m, 0, -1) + Uf(m, 0, 0), Wf(m - 3, 0, 0), Wf(m - 2, 0, 0), \
                       Wf(m - 1, 0, 0), Wf(m, 0, 0), Wf(m + 1, 0, 0), Wf(m + 2, 0, 0))
#define FWY(m) KL_FLUX(Vf(0, m, -1) + Vf(0, m, 0), Wf(0, m - 3, 0), Wf(0, m - 2, 0), \
                       Wf(0, m - 1, 0), Wf(0, m, 0), Wf(0, m + 1, 0), Wf(0, m + 2, 0))
#define FWZ(m) KL_FLUX(Wf(0, 0, m) + Wf(0, 0, m + 1), Wf(0, 0, m - 2), Wf(0, 0, m - 1), \
                       Wf(0, 0, m), Wf(0, 0, m + 1), Wf(0, 0, m + 2), Wf(0, 0, m + 3))

struct kl_coef {
    C cx, cy;       // KL_FS * dxi, KL_FS * dyi
    C dxi, dyi;
    C nux, nuy;     // nu * dxi^2, nu * dyi^2
    C nu;
};

// Tendencies of u, v, w at one point.  wall_w: w sits on a wall face (wt = 0).
template <class Acc>
__device__ __forceinline__ void kl_point(const Acc &A, const kl_coef &K, const kl_zmetric &Z,
                                         bool wall_w, C &tu, C &tv, C &tw)
{
    tu = C(0); tv = C(0); tw = C(0);
#if KL_ADV
    {
        C czu = KL_FS * Z.dzi, czw = KL_FS * Z.dzhi;
        tu = -((FUX(0) - FUX(-1)) * K.cx + (FUY(1) - FUY(0)) * K.cy + (FUZ(1) - FUZ(0)) * czu);
        tv = -((FVX(1) - FVX(0)) * K.cx + (FVY(0) - FVY(-1)) * K.cy + (FVZ(1) - FVZ(0)) * czu);
        tw = -((FWX(1) - FWX(0)) * K.cx + (FWY(1) - FWY(0)) * K.cy + (FWZ(0) - FWZ(-1)) * czw);
    }
#endif
#if KL_DIFF == 1
    {
        C u0 = Uf(0, 0, 0), v0 = Vf(0, 0, 0), w0 = Wf(0, 0, 0);
        tu += K.nux * (Uf(1, 0, 0) + Uf(-1, 0, 0) - C(2) * u0)
            + K.nuy * (Uf(0, 1, 0) + Uf(0, -1, 0) - C(2) * u0)
            + K.nu * ((Uf(0, 0, 1) - u0) * Z.dzhi_up - (u0 - Uf(0, 0, -1)) * Z.dzhi) * Z.dzi;
        tv += K.nux * (Vf(1, 0, 0) + Vf(-1, 0, 0) - C(2) * v0)
            + K.nuy * (Vf(0, 1, 0) + Vf(0, -1, 0) - C(2) * v0)
            + K.nu * ((Vf(0, 0, 1) - v0) * Z.dzhi_up - (v0 - Vf(0, 0, -1)) * Z.dzhi) * Z.dzi;
        tw += K.nux * (Wf(1, 0, 0) + Wf(-1, 0, 0) - C(2) * w0)
            + K.nuy * (Wf(0, 1, 0) + Wf(0, -1, 0) - C(2) * w0)
            + K.nu * ((Wf(0, 0, 1) - w0) * Z.dzi - (w0 - Wf(0, 0, -1)) * Z.dzi_dn) * Z.dzhi;
    }
#elif KL_DIFF == 2
    {
        const C q = C(0.25), two = C(2);
        const C dxi = K.dxi, dyi = K.dyi;
        // u point (xh_i, y_j, z_k)
        C sxx0 = two * Nf(0, 0, 0) * (Uf(1, 0, 0) - Uf(0, 0, 0)) * dxi;
        C sxx1 = two * Nf(-1, 0, 0) * (Uf(0, 0, 0) - Uf(-1, 0, 0)) * dxi;
        C nxy0 = q * (Nf(-1, -1, 0) + Nf(0, -1, 0) + Nf(-1, 0, 0) + Nf(0, 0, 0));
        C nxy1 = q * (Nf(-1, 0, 0) + Nf(0, 0, 0) + Nf(-1, 1, 0) + Nf(0, 1, 0));
        C sxy0 = nxy0 * ((Uf(0, 0, 0) - Uf(0, -1, 0)) * dyi + (Vf(0, 0, 0) - Vf(-1, 0, 0)) * dxi);
        C sxy1 = nxy1 * ((Uf(0, 1, 0) - Uf(0, 0, 0)) * dyi + (Vf(0, 1, 0) - Vf(-1, 1, 0)) * dxi);
        C nxz0 = q * (Nf(-1, 0, -1) + Nf(0, 0, -1) + Nf(-1, 0, 0) + Nf(0, 0, 0));
        C nxz1 = q * (Nf(-1, 0, 0) + Nf(0, 0, 0) + Nf(-1, 0, 1) + Nf(0, 0, 1));
        C sxz0 = nxz0 * ((Uf(0, 0, 0) - Uf(0, 0, -1)) * Z.dzhi + (Wf(0, 0, 0) - Wf(-1, 0, 0)) * dxi);
        C sxz1 = nxz1 * ((Uf(0, 0, 1) - Uf(0, 0, 0)) * Z.dzhi_up + (Wf(0, 0, 1) - Wf(-1, 0, 1)) * dxi);
        tu += (sxx0 - sxx1) * dxi + (sxy1 - sxy0) * dyi + (sxz1 - sxz0) * Z.dzi;
        // v point (x_i, yh_j, z_k)
        C nyx0 = q * (Nf(-1, -1, 0) + Nf(0, -1, 0) + Nf(-1, 0, 0) + Nf(0, 0, 0));
        C nyx1 = q * (Nf(0, -1, 0) + Nf(1, -1, 0) + Nf(0, 0, 0) + Nf(1, 0, 0));
        C syx0 = nyx0 * ((Vf(0, 0, 0) - Vf(-1, 0, 0)) * dxi + (Uf(0, 0, 0) - Uf(0, -1, 0)) * dyi);
        C syx1 = nyx1 * ((Vf(1, 0, 0) - Vf(0, 0, 0)) * dxi + (Uf(1, 0, 0) - Uf(1, -1, 0)) * dyi);
        C syy0 = two * Nf(0, 0, 0) * (Vf(0, 1, 0) - Vf(0, 0, 0)) * dyi;
        C syy1 = two * Nf(0, -1, 0) * (Vf(0, 0, 0) - Vf(0, -1, 0)) * dyi;
        C nyz0 = q * (Nf(0, -1, -1) + Nf(0, 0, -1) + Nf(0, -1, 0) + Nf(0, 0, 0));
        C nyz1 = q * (Nf(0, -1, 0) + Nf(0, 0, 0) + Nf(0, -1, 1) + Nf(0, 0, 1));
        C syz0 = nyz0 * ((Vf(0, 0, 0) - Vf(0, 0, -1)) * Z.dzhi + (Wf(0, 0, 0) - Wf(0, -1, 0)) * dyi);
        C syz1 = nyz1 * ((Vf(0, 0, 1) - Vf(0, 0, 0)) * Z.dzhi_up + (Wf(0, 0, 1) - Wf(0, -1, 1)) * dyi);
        tv += (syx1 - syx0) * dxi + (syy0 - syy1) * dyi + (syz1 - syz0) * Z.dzi;
        // w point (x_i, y_j, zh_k)
        C nzx0 = q * (Nf(-1, 0, -1) + Nf(0, 0, -1) + Nf(-1, 0, 0) + Nf(0, 0, 0));
        C nzx1 = q * (Nf(0, 0, -1) + Nf(1, 0, -1) + Nf(0, 0, 0) + Nf(1, 0, 0));
        C szx0 = nzx0 * ((Wf(0, 0, 0) - Wf(-1, 0, 0)) * dxi + (Uf(0, 0, 0) - Uf(0, 0, -1)) * Z.dzhi);
        C szx1 = nzx1 * ((Wf(1, 0, 0) - Wf(0, 0, 0)) * dxi + (Uf(1, 0, 0) - Uf(1, 0, -1)) * Z.dzhi);
        C nzy0 = q * (Nf(0, -1, -1) + Nf(0, 0, -1) + Nf(0, -1, 0) + Nf(0, 0, 0));
        C nzy1 = q * (Nf(0, 0, -1) + Nf(0, 1, -1) + Nf(0, 0, 0) + Nf(0, 1, 0));
        C szy0 = nzy0 * ((Wf(0, 0, 0) - Wf(0, -1, 0)) * dyi + (Vf(0, 0, 0) - Vf(0, 0, -1)) * Z.dzhi);
        C szy1 = nzy1 * ((Wf(0, 1, 0) - Wf(0, 0, 0)) * dyi + (Vf(0, 1, 0) - Vf(0, 1, -1)) * Z.dzhi);
        C szz0 = two * Nf(0, 0, 0) * (Wf(0, 0, 1) - Wf(0, 0, 0)) * Z.dzi;
        C szz1 = two * Nf(0, 0, -1) * (Wf(0, 0, 0) - Wf(0, 0, -1)) * Z.dzi_dn;
        tw += (szx1 - szx0) * dxi + (szy1 - szy0) * dyi + (szz0 - szz1) * Z.dzhi;
    }
#endif
    if (wall_w) tw = C(0);
}

__device__ __forceinline__ kl_coef kl_make_coef(const kl_args &a)
{
    kl_coef K;
    K.dxi = KL_CO(a, 0);
    K.dyi = KL_CO(a, 1);
    K.cx = KL_FS * K.dxi;
    K.cy = KL_FS * K.dyi;
    K.nu = KL_CO(a, 4);
    K.nux = KL_CO(a, 5);
    K.nuy = KL_CO(a, 6);
    return K;
}

__device__ __forceinline__ kl_zmetric kl_make_z(const kl_args &a, int k)
{
    kl_zmetric Z;
#if KL_ZUNI
    Z.dzi = Z.dzhi = Z.dzhi_up = Z.dzi_dn = KL_CO(a, 2);
#else
    Z.dzi = a.dzi[k];
    Z.dzhi = a.dzhi[k];
    Z.dzhi_up = a.dzhi[k + 1];
    Z.dzi_dn = a.dzi[k - 1];
#endif
    return Z;
}

#if KL_FAMILY == 0
// ======================================================= direct family
//
// One thread computes KL_TX x KL_TY x KL_TZ points; every neighbour is read
// from global memory through the read-only path.  When a tile is consecutive
// and unrolled, neighbouring points share loads and face fluxes by common
// subexpression elimination.

struct kl_acc_direct {
    const T *u, *v, *w, *n;
    int sj, sk;
    template <int a, int b, int c> __device__ __forceinline__ C U() const { return ld(u + (a + b * sj + c * sk)); }
    template <int a, int b, int c> __device__ __forceinline__ C V() const { return ld(v + (a + b * sj + c * sk)); }
    template <int a, int b, int c> __device__ __forceinline__ C W() const { return ld(w + (a + b * sj + c * sk)); }
    template <int a, int b, int c> __device__ __forceinline__ C N() const { return ld(n + (a + b * sj + c * sk)); }
};

#define KL_PRAGMA(x) _Pragma(#x)
#if KL_UX
#define KL_UNROLL_X KL_PRAGMA(unroll)
#else
#define KL_UNROLL_X KL_PRAGMA(unroll 1)
#endif
#if KL_UY
#define KL_UNROLL_Y KL_PRAGMA(unroll)
#else
#define KL_UNROLL_Y KL_PRAGMA(unroll 1)
#endif
#if KL_UZ
#define KL_UNROLL_Z KL_PRAGMA(unroll)
#else
#define KL_UNROLL_Z KL_PRAGMA(unroll 1)
#endif

template <bool FULL>
__device__ __forceinline__ void kl_direct_tile(const kl_args &a, const kl_coef &K, int i0, int j0, int k0)
{
    const int sj = (int)a.sj, sk = (int)a.sk;
    const int nx = (int)a.nx, ny = (int)a.ny, nz = (int)a.nz;
    KL_UNROLL_Z
    for (int c = 0; c < KL_TZ; ++c) {
        int k = KL_CZ ? k0 + c : k0 + c * KL_BZ;
        if (!FULL && k >= nz) continue;
        kl_zmetric Z = kl_make_z(a, k);
        KL_UNROLL_Y
        for (int b = 0; b < KL_TY; ++b) {
            int j = KL_CY ? j0 + b : j0 + b * KL_BY;
            if (!FULL && j >= ny) continue;
            KL_UNROLL_X
            for (int q = 0; q < KL_TX; ++q) {
                int i = KL_CX ? i0 + q : i0 + q * KL_BX;
                if (!FULL && i >= nx) continue;
                int o = i + j * sj + k * sk;
                kl_acc_direct A;
                A.u = a.u + o; A.v = a.v + o; A.w = a.w + o; A.n = a.nu + o;
                A.sj = sj; A.sk = sk;
                C tu, tv, tw;
                kl_point(A, K, Z, KL_ZBC == 1 && k == 0, tu, tv, tw);
                out(a.ut + o, tu);
                out(a.vt + o, tv);
                out(a.wt + o, tw);
            }
        }
    }
}

extern "C" __global__ void __launch_bounds__(KL_BX * KL_BY * KL_BZ, KL_MINB)
kl_tendency(const kl_args a)
{
    // unravel the 1D block index; the first letter of the order varies fastest
    long long b = blockIdx.x, bx, by, bz;
    const long long nbx = a.nbx, nby = a.nby, nbz = a.nbz;
    (void)nbx; (void)nby; (void)nbz;
#if KL_PERM == 0
    bx = b % nbx; b /= nbx; by = b % nby; bz = b / nby;
#elif KL_PERM == 1
    bx = b % nbx; b /= nbx; bz = b % nbz; by = b / nbz;
#elif KL_PERM == 2
    by = b % nby; b /= nby; bx = b % nbx; bz = b / nbx;
#elif KL_PERM == 3
    by = b % nby; b /= nby; bz = b % nbz; bx = b / nbz;
#elif KL_PERM == 4
    bz = b % nbz; b /= nbz; bx = b % nbx; by = b / nbx;
#else
    bz = b % nbz; b /= nbz; by = b % nby; bx = b / nby;
#endif
    const int i0 = (int)bx * (KL_BX * KL_TX) + (KL_CX ? threadIdx.x * KL_TX : threadIdx.x);
    const int j0 = (int)by * (KL_BY * KL_TY) + (KL_CY ? threadIdx.y * KL_TY : threadIdx.y);
    const int k0 = (int)bz * (KL_BZ * KL_TZ) + (KL_CZ ? threadIdx.z * KL_TZ : threadIdx.z);
    const kl_coef K = kl_make_coef(a);
    const int ix = KL_CX ? i0 + KL_TX - 1 : i0 + (KL_TX - 1) * KL_BX;
    const int jx = KL_CY ? j0 + KL_TY - 1 : j0 + (KL_TY - 1) * KL_BY;
    const int kx = KL_CZ ? k0 + KL_TZ - 1 : k0 + (KL_TZ - 1) * KL_BZ;
    if (ix < a.nx && jx < a.ny && kx < a.nz)
        kl_direct_tile<true>(a, K, i0, j0, k0);
    else
        kl_direct_tile<false>(a, K, i0, j0, k0);
}
#endif  // KL_FAMILY == 0
