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
//   KL_OF32    1: ut, vt, wt stored as f32 (16-bit storage only), 0: as KL_DTYPE
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
#ifndef KL_PK
#define KL_PK 1       // zpack: packed f32x2 arithmetic for f32 compute
#endif
#ifndef KL_YX
#define KL_YX 0       // zpack: 1 exchange y faces between warps through shared memory
                      // (a second barrier per level); 2 the same one level ahead
                      // with the side and tile-top faces (one barrier per level)
#endif
#ifndef KL_CS
#define KL_CS 0       // zpack: one warp group per tendency component
#endif
#ifndef KL_PE
#define KL_PE 0       // zpack: persistent CTAs over ranges of (tile, level) pairs
#endif
#if KL_CS && KL_YX
#error "KL_CS forms every y face in its own warp group; KL_YX must be 0"
#endif
#ifndef KL_BATCH
#define KL_BATCH 0    // 1: one launch over many grids through a device tile table
#endif
#ifndef KL_OF32
#define KL_OF32 0     // 1: tendencies stored as f32 (16-bit storage of the inputs)
#endif
#if KL_OF32 && KL_DTYPE < 2
#error "KL_OF32 applies to 16-bit storage"
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
#if KL_OF32
typedef float TO;     // storage of the tendencies
#else
typedef T TO;
#endif

// Kernel argument block; the host fills an identical struct (8-byte members).
struct kl_args {
    const T *u, *v, *w, *nu;      // pointers at interior point (0,0,0)
    TO *ut, *vt, *wt;
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
    long long wait_cycles;        // limit of one device wait, SM clock cycles
    long long flags;              // bit 0: x, y ghosts supplied by the caller (a block
                                  // of an x-y decomposition): read them from memory
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

// Global stores of tendencies for the ring families: plain st.global with no
// memory clobber.  The tendencies never alias the shared-memory planes, and
// without the clobber the compiler may keep plane values it has already
// loaded across these stores (a generic store would force it to load them
// again, since it could point into shared memory).
__device__ __forceinline__ void kl_stg_b64(void *p, unsigned long long v)
{
    asm volatile("{\n .reg .u64 g;\n cvta.to.global.u64 g, %0;\n st.global.b64 [g], %1;\n}" ::"l"(p), "l"(v));
}
__device__ __forceinline__ void kl_stg_b32(void *p, unsigned v)
{
    asm volatile("{\n .reg .u64 g;\n cvta.to.global.u64 g, %0;\n st.global.b32 [g], %1;\n}" ::"l"(p), "r"(v));
}
__device__ __forceinline__ void kl_stg_b16(void *p, unsigned short v)
{
    asm volatile("{\n .reg .u64 g;\n cvta.to.global.u64 g, %0;\n st.global.b16 [g], %1;\n}" ::"l"(p), "h"(v));
}
__device__ __forceinline__ void kl_stg_v2f32(void *p, float a, float b)
{
    asm volatile("{\n .reg .u64 g;\n cvta.to.global.u64 g, %0;\n st.global.v2.f32 [g], {%1, %2};\n}"
                 ::"l"(p), "f"(a), "f"(b));
}
__device__ __forceinline__ void kl_stg_v2f64(void *p, double a, double b)
{
    asm volatile("{\n .reg .u64 g;\n cvta.to.global.u64 g, %0;\n st.global.v2.f64 [g], {%1, %2};\n}"
                 ::"l"(p), "d"(a), "d"(b));
}
__device__ __forceinline__ void kl_stg_f64(void *p, double v)
{
    asm volatile("{\n .reg .u64 g;\n cvta.to.global.u64 g, %0;\n st.global.f64 [g], %1;\n}" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void kl_stg_f32(void *p, float v)
{
    asm volatile("{\n .reg .u64 g;\n cvta.to.global.u64 g, %0;\n st.global.f32 [g], %1;\n}" ::"l"(p), "f"(v));
}

#if KL_OF32
__device__ __forceinline__ void out(TO *p, C v)
{
#if KL_ACC
    v += *p;
#endif
    *p = v;
}
#else
__device__ __forceinline__ void out(T *p, C v)
{
#if KL_ACC
    v += lds(p);
#endif
    st(p, v);
}
#endif

// one tendency value through the plain global stores above
__device__ __forceinline__ void outg(TO *p, C v)
{
#if KL_OF32
#if KL_ACC
    v += *p;
#endif
    kl_stg_f32(p, v);
#else
#if KL_ACC
    v += lds(p);
#endif
#if KL_DTYPE == 0
    kl_stg_f64(p, v);
#elif KL_DTYPE == 1
    kl_stg_f32(p, v);
#else
    kl_u16 r;
    st(&r, v);
    kl_stg_b16(p, r);
#endif
#endif
}

// ------------------------------------------------------------ face fluxes
//
// Us is twice the advecting velocity (sum of two neighbours); a0..a5 are the
// advected values around the face (face between a2 and a3).  The returned
// flux is scaled by KL_FS_INV; the caller multiplies by KL_FS.
//   5th order: 120 F = Us*(37(a2+a3) - 8(a1+a4) + (a0+a5))
//                     + |Us|*(10(a2-a3) - 5(a1-a4) + (a0-a5))
//   2nd order:   4 F = Us*(a2+a3)

// I6 keeps a2 and a3 unrounded until they are scaled by 37 (fused into the
// last two steps): rounding the pair sum a2 + a3 first would multiply its
// error by 37, making the face value's rounding error ~2.8 units instead of
// ~1.9, and the flux differences amplify that error by 1/(k dx).
__device__ __forceinline__ C flux5(C Us, C a0, C a1, C a2, C a3, C a4, C a5)
{
    C s2 = a1 + a4, s3 = a0 + a5;
    C d1 = a2 - a3, d2 = a1 - a4, d3 = a0 - a5;
    C i6 = fma(C(37), a2, fma(C(37), a3, fma(C(-8), s2, s3)));
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
// Vertical advective fluxes of the point's column: the bottom ones (faces
// below u, v and the centre below w) and the top ones.  A z-marching kernel
// carries the top fluxes of level k as the bottom fluxes of level k+1.
template <class Acc>
__device__ __forceinline__ void kl_zflux_bottom(const Acc &A, C f[3])
{
#if KL_ADV
    f[0] = FUZ(0); f[1] = FVZ(0); f[2] = FWZ(-1);
#else
    f[0] = f[1] = f[2] = C(0);
#endif
}

template <class Acc>
__device__ __forceinline__ void kl_zflux_top(const Acc &A, C f[3])
{
#if KL_ADV
    f[0] = FUZ(1); f[1] = FVZ(1); f[2] = FWZ(0);
#else
    f[0] = f[1] = f[2] = C(0);
#endif
}

// Tendencies of u, v, w at one point given its vertical fluxes (zb bottom,
// zt top).  wall_w: w sits on a wall face (wt = 0).
template <class Acc>
__device__ __forceinline__ void kl_point_z(const Acc &A, const kl_coef &K, const kl_zmetric &Z,
                                           const C zb[3], const C zt[3], bool wall_w,
                                           C &tu, C &tv, C &tw)
{
    tu = C(0); tv = C(0); tw = C(0);
#if KL_ADV
    {
        C czu = KL_FS * Z.dzi, czw = KL_FS * Z.dzhi;
        tu = -((FUX(0) - FUX(-1)) * K.cx + (FUY(1) - FUY(0)) * K.cy + (zt[0] - zb[0]) * czu);
        tv = -((FVX(1) - FVX(0)) * K.cx + (FVY(0) - FVY(-1)) * K.cy + (zt[1] - zb[1]) * czu);
        tw = -((FWX(1) - FWX(0)) * K.cx + (FWY(1) - FWY(0)) * K.cy + (zt[2] - zb[2]) * czw);
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

template <class Acc>
__device__ __forceinline__ void kl_point(const Acc &A, const kl_coef &K, const kl_zmetric &Z,
                                         bool wall_w, C &tu, C &tv, C &tw)
{
    C zb[3], zt[3];
    kl_zflux_bottom(A, zb);
    kl_zflux_top(A, zt);
    kl_point_z(A, K, Z, zb, zt, wall_w, tu, tv, tw);
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

__device__ __forceinline__ void kl_direct_block(const kl_args &a, long long b)
{
    // unravel the 1D block index; the first letter of the order varies fastest
    long long bx, by, bz;
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

#if KL_BATCH
// many grids in one launch: block b runs block blocks[b].y of grid blocks[b].x
extern "C" __global__ void __launch_bounds__(KL_BX * KL_BY * KL_BZ, KL_MINB)
kl_tendency(const kl_args *argv, const int4 *blocks)
{
    const int4 d = blocks[blockIdx.x];
    const kl_args a = argv[d.x];
    kl_direct_block(a, d.y);
}
#else
extern "C" __global__ void __launch_bounds__(KL_BX * KL_BY * KL_BZ, KL_MINB)
kl_tendency(const kl_args a)
{
    kl_direct_block(a, blockIdx.x);
}
#endif
#endif  // KL_FAMILY == 0

#if KL_FAMILY >= 1
// ================================= TMA plane ring shared by families 1 and 2

// A CTA of KL_MBX x KL_MBY threads owns an x-y tile of TXS x TYS interior
// points (each thread KL_MPX consecutive x points times KL_MPY consecutive
// rows) and marches up KL_KC levels.  Whole planes of the tile plus its
// in-plane halo are streamed into a ring of KL_NS shared-memory slots by TMA
// (one elected thread issues cp.async.bulk.tensor per field and plane; an
// mbarrier per slot counts the bytes).  Level k reads planes k-R .. k+R from
// the ring; its top vertical fluxes are kept in registers as the bottom
// fluxes of level k+1, and the x / y fluxes that neighbouring points of the
// same thread share are formed once (common subexpressions of identical
// shared-memory loads).  Every wait is bounded: on time-out the CTA records
// KL_DEV_TIMEOUT in the status word, drains its outstanding copies (again
// bounded) and returns.

#define KL_R (KL_ADV == 5 ? 3 : 1)                  // vertical reach
#define KL_H (KL_ADV == 5 ? 3 : 1)                  // in-plane halo
#define KL_AL (16 / (int)sizeof(T))                 // TMA x alignment, elements
#define KL_RUP(a, b) (((a) + (b) - 1) / (b) * (b))
#define KL_LPAD KL_RUP(KL_H, KL_AL)
#define KL_TXS (KL_MBX * KL_MPX)
#define KL_TYS (KL_MBY * KL_MPY)
#define KL_PITCH KL_RUP(KL_LPAD + KL_TXS + KL_H, KL_AL)
#define KL_ROWS (KL_TYS + 2 * KL_H)
#define KL_BOX_BYTES (KL_PITCH * KL_ROWS * (int)sizeof(T))
#define KL_PLANE_BYTES KL_RUP(KL_BOX_BYTES, 128)
#define KL_NF (KL_DIFF == 2 ? 4 : 3)
#define KL_SLOT_BYTES (KL_PLANE_BYTES * KL_NF)
#define KL_DEV_TIMEOUT 1
#define KL_WAIT_LIMIT (1 << 22)

static_assert(KL_NS >= 2 * KL_R + 2 || (KL_FAMILY == 2 && KL_NS >= 2 * KL_R),
              "ring must hold the stencil planes plus one in flight");
static_assert(KL_PITCH <= 256 && KL_ROWS <= 256, "TMA box dimension above 256");

struct __align__(64) kl_tmap { unsigned long long v[16]; };

__device__ __forceinline__ unsigned kl_smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void kl_mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void kl_mbar_expect(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool kl_mbar_try(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// non-blocking probe of the phase
__device__ __forceinline__ bool kl_mbar_test(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// bounded waits (iteration cap and a clock64 deadline).  The default build
// waits with try_wait up to 2^31 cycles, about one second.  A context whose
// wait limit was changed (kl_set_wait_limit) compiles its kernels with
// KL_WAITPOLL=1: the compute waits then poll with the non-blocking test_wait
// against the limit in the kernel arguments (try_wait may suspend on its
// own).  kl_mbar_drain, the wait for copies still in flight before a CTA
// leaves, always uses the default deadline.  Both return false on time-out.
#ifndef KL_WAITPOLL
#define KL_WAITPOLL 0
#endif
#define KL_DRAIN_CYCLES (1ll << 31)
__device__ __forceinline__ bool kl_mbar_drain(unsigned bar, unsigned parity)
{
    long long t0 = clock64();
    for (int it = 0; it < KL_WAIT_LIMIT; ++it) {
        if (kl_mbar_try(bar, parity)) return true;
        if (clock64() - t0 > KL_DRAIN_CYCLES) break;
    }
    return false;
}

__device__ __forceinline__ bool kl_mbar_wait(unsigned bar, unsigned parity, long long cycles)
{
#if KL_WAITPOLL
    long long t0 = clock64();
    for (int it = 0; it < KL_WAIT_LIMIT; ++it) {
        if (kl_mbar_test(bar, parity)) return true;
        if (clock64() - t0 > cycles) break;
    }
    return false;
#else
    (void)cycles;
    return kl_mbar_drain(bar, parity);
#endif
}

// a descriptor read from global memory (batched launches) is ordered after
// the host's copy of it for the tensor-map proxy by this fence
__device__ __forceinline__ void kl_tmap_acquire(const kl_tmap *m)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;"
                 ::"l"((unsigned long long)m) : "memory");
}

__device__ __forceinline__ void kl_tma_load3(unsigned dst, const kl_tmap *map, int x, int y, int z,
                                             unsigned bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(dst), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(bar)
                 : "memory");
}

#endif  // KL_FAMILY >= 1

#if KL_FAMILY == 1
// ======================================================= zmarch family
//
// (described above: one thread per KL_MPX x KL_MPY points, every stencil
// value read from the plane ring)

struct kl_acc_smem {
    const char *base[2 * KL_R + 1];     // slot base of plane k+dk, dk = -R..R
    int off;                            // byte offset of the point inside a plane
    template <int a, int b, int c> __device__ __forceinline__ C at(int f) const
    {
        static_assert(a >= -KL_H && a <= KL_H && b >= -KL_H && b <= KL_H, "offset outside the halo");
        static_assert(c >= -KL_R && c <= KL_R, "offset outside the staged planes");
        return lds((const T *)(base[c + KL_R] + f * KL_PLANE_BYTES + off +
                               (a + b * KL_PITCH) * (int)sizeof(T)));
    }
    template <int a, int b, int c> __device__ __forceinline__ C U() const { return at<a, b, c>(0); }
    template <int a, int b, int c> __device__ __forceinline__ C V() const { return at<a, b, c>(1); }
    template <int a, int b, int c> __device__ __forceinline__ C W() const { return at<a, b, c>(2); }
    template <int a, int b, int c> __device__ __forceinline__ C N() const { return at<a, b, c>(3); }
};

__device__ __forceinline__ void kl_zmarch_body(const kl_args &a, const kl_tmap *const *maps,
                                               int bxi, int byi, int bzi)
{
    extern __shared__ unsigned char kl_smem_raw[];
    unsigned char *ring = (unsigned char *)(((unsigned long long)kl_smem_raw + 127) & ~127ull);
    unsigned long long *bars = (unsigned long long *)(ring + KL_NS * KL_SLOT_BYTES);
    const int tid = threadIdx.x + threadIdx.y * KL_MBX;
    const int nx = (int)a.nx, ny = (int)a.ny, nz = (int)a.nz;
    const int kb = bzi * (int)a.kchunk;
    const int ke = min(kb + (int)a.kchunk, nz);
    const int tx0 = bxi * KL_TXS, ty0 = byi * KL_TYS;
    const int gx = (int)a.tile_x0 + tx0 - KL_LPAD, gy = (int)a.tile_y0 + ty0 - KL_H;
    const int gz0 = (int)a.tile_z0;

    if (tid == 0) {
        for (int s = 0; s < KL_NS; ++s) kl_mbar_init(kl_smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // plane p (interior level) lives in ring slot (p - (kb - R)) mod NS
    auto issue = [&](int p) {
        int slot = (p - (kb - KL_R)) % KL_NS;
        unsigned bar = kl_smem_addr(&bars[slot]);
        kl_mbar_expect(bar, KL_NF * KL_BOX_BYTES);
        unsigned dst = kl_smem_addr(ring + slot * KL_SLOT_BYTES);
#pragma unroll
        for (int f = 0; f < KL_NF; ++f)
            kl_tma_load3(dst + f * KL_PLANE_BYTES, maps[f], gx, gy, gz0 + p, bar);
    };
    const int p_first = kb - KL_R;
    const int p_last = ke - 1 + KL_R;                 // last plane this CTA needs
    int p_next = p_first;                             // next plane to issue
    if (tid == 0)
        for (; p_next < p_first + KL_NS && p_next <= p_last; ++p_next) issue(p_next);

    const kl_coef K = kl_make_coef(a);
    const int lx = KL_LPAD + threadIdx.x * KL_MPX;
    const int ly = KL_H + threadIdx.y * KL_MPY;
    C zb[KL_MPY][KL_MPX][3];
    bool timed_out = false;
    int p_waited = p_first - 1;                       // every plane <= this has landed

    for (int k = kb; k < ke; ++k) {
        // the newest plane this level needs is k + R
        {
            int p = k + KL_R;
            int use = (p - p_first) / KL_NS;
            unsigned bar = kl_smem_addr(&bars[(p - p_first) % KL_NS]);
            // at the first level also the planes below must have landed
            if (k == kb) {
                for (int q = p_first; q < p; ++q) {
                    unsigned b2 = kl_smem_addr(&bars[(q - p_first) % KL_NS]);
                    bool ok2 = kl_mbar_wait(b2, ((q - p_first) / KL_NS) & 1, a.wait_cycles);
                    if (__syncthreads_or(!ok2)) { timed_out = true; break; }
                    p_waited = q;
                }
                if (timed_out) break;
            }
            bool ok = kl_mbar_wait(bar, use & 1, a.wait_cycles);
            if (__syncthreads_or(!ok)) { timed_out = true; break; }
            p_waited = p;
        }
        kl_acc_smem A;
#pragma unroll
        for (int d = -KL_R; d <= KL_R; ++d)
            A.base[d + KL_R] = (const char *)(ring + ((k + d - p_first) % KL_NS) * KL_SLOT_BYTES);
        const kl_zmetric Z = kl_make_z(a, k);
        const int k_out = k;
#pragma unroll
        for (int r = 0; r < KL_MPY; ++r) {
#pragma unroll
            for (int q = 0; q < KL_MPX; ++q) {
                A.off = ((ly + r) * KL_PITCH + lx + q) * (int)sizeof(T);
                C zt[3];
                if (k == kb) kl_zflux_bottom(A, zb[r][q]);
                kl_zflux_top(A, zt);
                C tu, tv, tw;
                kl_point_z(A, K, Z, zb[r][q], zt, KL_ZBC == 1 && k_out == 0, tu, tv, tw);
                zb[r][q][0] = zt[0];
                zb[r][q][1] = zt[1];
                zb[r][q][2] = zt[2];
                const int i = tx0 + threadIdx.x * KL_MPX + q;
                const int j = ty0 + threadIdx.y * KL_MPY + r;
                if (i < nx && j < ny) {
                    long long o = i + (long long)j * a.sj + (long long)k_out * a.sk;
                    out(a.ut + o, tu);
                    out(a.vt + o, tv);
                    out(a.wt + o, tw);
                }
            }
        }
        // every thread is done with plane k - R: refill its slot
        __syncthreads();
        if (tid == 0 && p_next <= p_last) issue(p_next++);
    }

    if (timed_out) {
        if (tid == 0) {
            atomicOr(a.err, KL_DEV_TIMEOUT);
            // drain: wait (bounded) for the copies still in flight before
            // leaving, so no TMA write lands in shared memory after exit
            for (int q = p_waited + 1; q < p_next; ++q) {
                unsigned b2 = kl_smem_addr(&bars[(q - p_first) % KL_NS]);
                kl_mbar_drain(b2, ((q - p_first) / KL_NS) & 1);
            }
        }
        __syncthreads();
    }
}

#if KL_BATCH
// many grids in one launch: block b runs tile (y, z, w) of grid x of blocks[b];
// TMA descriptors of grid g at maps[7g .. 7g+3] (global memory, 64-B aligned)
extern "C" __global__ void __launch_bounds__(KL_MBX * KL_MBY, KL_MMINB)
kl_tendency(const kl_args *argv, const int4 *blocks, const kl_tmap *tmaps)
{
    const int4 d = blocks[blockIdx.x];
    const kl_args a = argv[d.x];
    const kl_tmap *maps[4] = {&tmaps[7 * d.x], &tmaps[7 * d.x + 1], &tmaps[7 * d.x + 2],
                              &tmaps[7 * d.x + 3]};
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int f = 0; f < KL_NF; ++f) kl_tmap_acquire(maps[f]);
    kl_zmarch_body(a, maps, d.y, d.z, d.w);
}
#else
extern "C" __global__ void __launch_bounds__(KL_MBX * KL_MBY, KL_MMINB)
kl_tendency(const kl_args a, const __grid_constant__ kl_tmap tm_u,
            const __grid_constant__ kl_tmap tm_v, const __grid_constant__ kl_tmap tm_w,
            const __grid_constant__ kl_tmap tm_n)
{
    const kl_tmap *maps[4] = {&tm_u, &tm_v, &tm_w, &tm_n};
    kl_zmarch_body(a, maps, blockIdx.x, blockIdx.y, blockIdx.z);
}
#endif
#endif  // KL_FAMILY == 1

#if KL_FAMILY == 2
// ======================================================== zpack family
//
// Same plane ring as zmarch (tile 64 x KL_TYS, KL_MBY warps, each warp KL_MPY
// consecutive rows); every face flux is formed once and diffusion is folded
// into it:
//  * lane l of a warp owns the two adjacent columns c0 = x0 + 2l, c1 = c0 + 1
//    as one packed value (f32x2 for f32 compute, two doubles for f64); an
//    aligned pair is one 8-byte (f32) shared load that lands in the packed
//    register, odd offsets are formed from two aligned pairs, and results are
//    stored with one vector store per field;
//  * x: a lane forms the faces of both its columns on one side and gets the
//    face on the other side of the pair from its neighbour lane by a shuffle;
//    the one face per row beyond the warp's 64 columns is formed for all rows
//    of the warp in one side pass (lane e: field e / MPY, row e % MPY);
//  * y: a thread's consecutive rows share their faces (two live per field);
//  * z: the top face of level k is carried as the bottom face of level k+1;
//  * constant-nu diffusion: the diffusive flux nu (a_{m+1} - a_m) / d of a face
//    is added to the advective flux of the same face, using the difference
//    d1 = a_m - a_{m+1} the upwind formula already forms;
//  * variable-nu diffusion (stress form): each face flux gets its stress
//    -S / FS; a shear stress on an edge (xy, xz, yz) is formed once and used
//    by both components that share the edge (u's y face and v's x face, u's
//    z face and w's x face, v's z face and w's y face), the z-edge stresses
//    carried from one level to the next like the z fluxes; nu streams
//    through its own ring of planes k-1 .. k+1 (rows -1 .. TYS of the tile).

#if KL_DTYPE == 0 || KL_PK == 0
// two independent scalars (f64, or f32 with packed arithmetic switched off)
struct V { C lo, hi; };
__device__ __forceinline__ V vmk(C a, C b) { V r; r.lo = a; r.hi = b; return r; }
__device__ __forceinline__ C vlo(V a) { return a.lo; }
__device__ __forceinline__ C vhi(V a) { return a.hi; }
__device__ __forceinline__ V vadd(V a, V b) { return vmk(a.lo + b.lo, a.hi + b.hi); }
__device__ __forceinline__ V vsub(V a, V b) { return vmk(a.lo - b.lo, a.hi - b.hi); }
__device__ __forceinline__ V vmul(V a, V b) { return vmk(a.lo * b.lo, a.hi * b.hi); }
__device__ __forceinline__ V vfma(V a, V b, V c) { return vmk(fma(a.lo, b.lo, c.lo), fma(a.hi, b.hi, c.hi)); }
#if KL_DTYPE == 0
// aligned pair of consecutive elements at p (16-byte aligned)
__device__ __forceinline__ V vld(const T *p) { double2 d = *(const double2 *)p; return vmk(d.x, d.y); }
__device__ __forceinline__ void vst(T *p, V a) { kl_stg_v2f64(p, a.lo, a.hi); }
#elif KL_DTYPE == 1
__device__ __forceinline__ V vld(const T *p) { float2 d = *(const float2 *)p; return vmk(d.x, d.y); }
__device__ __forceinline__ void vst(T *p, V a) { kl_stg_v2f32(p, a.lo, a.hi); }
#else
__device__ __forceinline__ V vld(const T *p)
{
    unsigned w = *(const unsigned *)p;
    kl_u16 lo = (kl_u16)(w & 0xffffu), hi = (kl_u16)(w >> 16);
    return vmk(lds(&lo), lds(&hi));
}
__device__ __forceinline__ void vst(T *p, V a)
{
    kl_u16 lo, hi;
    st(&lo, a.lo);
    st(&hi, a.hi);
    kl_stg_b32(p, (unsigned)lo | ((unsigned)hi << 16));
}
#endif
__device__ __forceinline__ V vldg(const T *p) { return vld(p); }
#else
struct V { unsigned long long b; };
__device__ __forceinline__ V vmk(float a, float c)
{
    V r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.b) : "f"(a), "f"(c));
    return r;
}
__device__ __forceinline__ float vlo(V a)
{
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.b));
    return lo;
}
__device__ __forceinline__ float vhi(V a)
{
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.b));
    return hi;
}
__device__ __forceinline__ V vadd(V a, V b) { V r; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(b.b)); return r; }
__device__ __forceinline__ V vsub(V a, V b) { V r; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(b.b)); return r; }
__device__ __forceinline__ V vmul(V a, V b) { V r; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(b.b)); return r; }
__device__ __forceinline__ V vfma(V a, V b, V c)
{
    V r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.b) : "l"(a.b), "l"(b.b), "l"(c.b));
    return r;
}
#if KL_DTYPE == 1
__device__ __forceinline__ V vld(const T *p) { V r; r.b = *(const unsigned long long *)p; return r; }
__device__ __forceinline__ void vst(T *p, V a) { kl_stg_b64(p, a.b); }
#else
// two 16-bit values in one 32-bit word, widened to f32
__device__ __forceinline__ V vld(const T *p)
{
    unsigned w = *(const unsigned *)p;
    kl_u16 lo = (kl_u16)(w & 0xffffu), hi = (kl_u16)(w >> 16);
    return vmk(lds(&lo), lds(&hi));
}
__device__ __forceinline__ void vst(T *p, V a)
{
    kl_u16 lo, hi;
    st(&lo, vlo(a));
    st(&hi, vhi(a));
    kl_stg_b32(p, (unsigned)lo | ((unsigned)hi << 16));
}
#endif
__device__ __forceinline__ V vldg(const T *p) { return vld(p); }
#endif
__device__ __forceinline__ V vsplat(C a) { return vmk(a, a); }
// aligned pair of tendencies (outputs): the storage type, or f32 (KL_OF32)
#if KL_OF32
__device__ __forceinline__ void vsto(TO *p, V a) { kl_stg_v2f32(p, vlo(a), vhi(a)); }
__device__ __forceinline__ V vldo(const TO *p) { float2 d = *(const float2 *)p; return vmk(d.x, d.y); }
#else
__device__ __forceinline__ void vsto(TO *p, V a) { vst(p, a); }
__device__ __forceinline__ V vldo(const TO *p) { return vldg(p); }
#endif
// (hi of a, lo of b): the pair starting one element after a's
__device__ __forceinline__ V vcross(V a, V b) { return vmk(vhi(a), vlo(b)); }

struct kl_vk { V c37, cm8, c10, cm5, cm10, c5; };

// packed face flux with the diffusive part folded in:
//   G = F + kd * d1,  F as flux5 / flux2 (scaled by 1/KL_FS), d1 = a2 - a3
__device__ __forceinline__ V kl_vflux(const kl_vk &K, V Us, V a0, V a1, V a2, V a3, V a4, V a5, V kd)
{
    V d1 = vsub(a2, a3);
#if KL_ADV == 5
    // a2, a3 stay unrounded until scaled by 37 (see flux5)
    V s2 = vadd(a1, a4), s3 = vadd(a0, a5);
    V d2 = vsub(a1, a4), d3 = vsub(a0, a5);
    V i6 = vfma(K.c37, a2, vfma(K.c37, a3, vfma(K.cm8, s2, s3)));
    V d6 = vfma(K.c10, d1, vfma(K.cm5, d2, d3));
    // |U| d6 as two scalar products: the absolute value folds into the
    // multiply as an operand modifier instead of two integer masks
    V f = vfma(Us, i6, vmk(fabs(vlo(Us)) * vlo(d6), fabs(vhi(Us)) * vhi(d6)));
#elif KL_ADV == 2
    V f = vmul(Us, vadd(a2, a3));
#else
    V f = vsplat(C(0));
#endif
#if KL_DIFF == 1
    f = vfma(kd, d1, f);
#endif
    return f;
}

// scalar twin for the side pass
__device__ __forceinline__ C kl_sflux(C Us, C a0, C a1, C a2, C a3, C a4, C a5, C kd)
{
    C d1 = a2 - a3;
#if KL_ADV == 5
    C f = flux5(Us, a0, a1, a2, a3, a4, a5);
#elif KL_ADV == 2
    C f = flux2(Us, a2, a3);
#else
    C f = C(0);
#endif
#if KL_DIFF == 1
    f = fma(kd, d1, f);
#endif
    return f;
}

// the 4 outer values of a 6-point window exist only for the 5th-order scheme;
// other schemes never address them (their planes / rows lie outside the ring)
#if KL_ADV == 5
#define KL_A5(x) (x)
#else
#define KL_A5(x) vsplat(C(0))
#endif

#define KL_OFF(x, row) ((((row) + KL_H) * KL_PITCH + (x)) * (int)sizeof(T))

// aligned pair of field F on plane k+DK at columns (lx + DX, lx + DX + 1),
// tile row `row`; DX even (lx is even), offsets checked at compile time
template <int F, int DK, int DX>
__device__ __forceinline__ V kl_pr(const char *const *pl, int lx, int row)
{
    static_assert(DK >= -KL_R && DK <= KL_R, "plane outside the staged window");
    static_assert(DX % 2 == 0, "pairs start on even columns");
    // lx ranges over [LPAD, LPAD + 62]: the pair must stay inside [0, PITCH)
    static_assert(DX >= -KL_LPAD && KL_LPAD + 62 + DX + 1 < KL_PITCH, "x offset outside the box");
    static_assert(F >= 0 && F < 3, "field index");
    return vld((const T *)(pl[DK + KL_R] + F * KL_PLANE_BYTES + KL_OFF(lx + DX, row)));
}

#if KL_CS
// ---- component split (cs=1): the block holds three groups of KL_MBY warps
// over the same tile; group CP forms every face flux of tendency component CP
// (0: u, 1: v, 2: w) with the same expressions, in the same order, as the
// all-component path, so both give identical results.  A thread carries one
// component's z faces instead of three, which leaves room for three times the
// warps per tile.
#define KL_P(f, dk, dx, row) kl_pr<(f), (dk), (dx)>(pl, lx, (row))

// y face of component CP at the bottom edge of tile row yr
template <int CP>
__device__ __forceinline__ V kl_cs_yface(const kl_vk &K, const char *const *pl, int lx, int yr, V kd)
{
    V us;
    if constexpr (CP == 0) us = vadd(vcross(KL_P(1, 0, -2, yr), KL_P(1, 0, 0, yr)), KL_P(1, 0, 0, yr));
    else if constexpr (CP == 1) us = vadd(KL_P(1, 0, 0, yr - 1), KL_P(1, 0, 0, yr));
    else us = vadd(KL_P(1, -1, 0, yr), KL_P(1, 0, 0, yr));
    return kl_vflux(K, us, KL_A5(KL_P(CP, 0, 0, yr - 3)), KL_A5(KL_P(CP, 0, 0, yr - 2)),
                    KL_P(CP, 0, 0, yr - 1), KL_P(CP, 0, 0, yr), KL_A5(KL_P(CP, 0, 0, yr + 1)),
                    KL_A5(KL_P(CP, 0, 0, yr + 2)), kd);
}

// z face of component CP below plane DK (DK = 1: top face of the level, 0: bottom)
template <int CP, int DK>
__device__ __forceinline__ V kl_cs_zface(const kl_vk &K, const char *const *pl, int lx, int yr, V kd)
{
    V us;
    if constexpr (CP == 0) us = vadd(vcross(KL_P(2, DK, -2, yr), KL_P(2, DK, 0, yr)), KL_P(2, DK, 0, yr));
    else if constexpr (CP == 1) us = vadd(KL_P(2, DK, 0, yr - 1), KL_P(2, DK, 0, yr));
    else us = vadd(KL_P(2, DK - 1, 0, yr), KL_P(2, DK, 0, yr));
    return kl_vflux(K, us, KL_A5(KL_P(CP, DK - 3, 0, yr)), KL_A5(KL_P(CP, DK - 2, 0, yr)),
                    KL_P(CP, DK - 1, 0, yr), KL_P(CP, DK, 0, yr), KL_A5(KL_P(CP, DK + 1, 0, yr)),
                    KL_A5(KL_P(CP, DK + 2, 0, yr)), kd);
}

template <int CP>
__device__ __forceinline__ void kl_cs_level(const kl_args &a, const kl_vk &K, const char *const *pl,
                                            const kl_zmetric &Z, int lane, int lx, int r0, int c0,
                                            int ty0, int k, int kb, C nu, C kdx, V vkdx, V vkdy,
                                            V vcx, V vcy, V (&zb)[KL_MPY])
{
    const V vcz = vsplat(KL_FS * (CP == 2 ? Z.dzhi : Z.dzi));
    const V vkz_top = vsplat(nu * (CP == 2 ? Z.dzi : Z.dzhi_up) / KL_FS);

    // side pass: lane e < KL_MPY forms the x face beyond the warp's columns of row r0 + e
    C extra;
    {
        const int row = r0 + (lane < KL_MPY ? lane : 0);
        const int xs = CP == 0 ? KL_LPAD - 3 : KL_LPAD + 61;
        const char *base = pl[KL_R] + CP * KL_PLANE_BYTES;
        C a2 = lds((const T *)(base + KL_OFF(xs + 2, row)));
        C a3 = lds((const T *)(base + KL_OFF(xs + 3, row)));
#if KL_ADV == 5
        C a0 = lds((const T *)(base + KL_OFF(xs, row)));
        C a1 = lds((const T *)(base + KL_OFF(xs + 1, row)));
        C a4 = lds((const T *)(base + KL_OFF(xs + 4, row)));
        C a5 = lds((const T *)(base + KL_OFF(xs + 5, row)));
#else
        C a0 = C(0), a1 = C(0), a4 = C(0), a5 = C(0);
#endif
        C us;
        if constexpr (CP == 0)
            us = a2 + a3;
        else if constexpr (CP == 1)
            us = lds((const T *)(pl[KL_R] + KL_OFF(KL_LPAD + 64, row - 1))) +
                 lds((const T *)(pl[KL_R] + KL_OFF(KL_LPAD + 64, row)));
        else
            us = lds((const T *)(pl[KL_R - 1] + KL_OFF(KL_LPAD + 64, row))) +
                 lds((const T *)(pl[KL_R] + KL_OFF(KL_LPAD + 64, row)));
        extra = kl_sflux(us, a0, a1, a2, a3, a4, a5, kdx);
    }

    V fy_b = kl_cs_yface<CP>(K, pl, lx, r0, vkdy);
    TO *const dst = CP == 0 ? a.ut : CP == 1 ? a.vt : a.wt;
#pragma unroll
    for (int r = 0; r < KL_MPY; ++r) {
        const int yr = r0 + r;
        // x faces of both columns; the face on the far side of the pair comes
        // from the neighbour lane, or from the side pass at the warp's edge
        const C e = __shfl_sync(0xffffffffu, extra, r);
        V tx;
        if constexpr (CP == 0) {
            V u_m2 = KL_A5(KL_P(0, 0, -2, yr)), u_0 = KL_P(0, 0, 0, yr), u_2 = KL_P(0, 0, 2, yr);
            V fx = kl_vflux(K, vadd(u_0, vcross(u_0, u_2)), KL_A5(u_m2), KL_A5(vcross(u_m2, u_0)), u_0,
                            vcross(u_0, u_2), KL_A5(u_2), KL_A5(vcross(u_2, KL_P(0, 0, 4, yr))), vkdx);
            C hi = __shfl_sync(0xffffffffu, vhi(fx), (lane + 31) & 31);
            tx = vsub(vmk(lane == 0 ? e : hi, vlo(fx)), fx);
        } else {
            V m4 = KL_A5(KL_P(CP, 0, -4, yr)), m2 = KL_P(CP, 0, -2, yr), p0 = KL_P(CP, 0, 0, yr),
              p2 = KL_P(CP, 0, 2, yr);
            V us = CP == 1 ? vadd(KL_P(0, 0, 0, yr - 1), KL_P(0, 0, 0, yr))
                           : vadd(KL_P(0, -1, 0, yr), KL_P(0, 0, 0, yr));
            V fx = kl_vflux(K, us, KL_A5(vcross(m4, m2)), KL_A5(m2), vcross(m2, p0), p0,
                            KL_A5(vcross(p0, p2)), KL_A5(p2), vkdx);
            C lo = __shfl_sync(0xffffffffu, vlo(fx), (lane + 1) & 31);
            tx = vsub(fx, vmk(vhi(fx), lane == 31 ? e : lo));
        }
        const V fy_t = kl_cs_yface<CP>(K, pl, lx, yr + 1, vkdy);
        const V fz = kl_cs_zface<CP, 1>(K, pl, lx, yr, vkz_top);
        if (k == kb)
            zb[r] = kl_cs_zface<CP, 0>(K, pl, lx, yr,
                                       vsplat(nu * (CP == 2 ? Z.dzi_dn : Z.dzhi) / KL_FS));
        V t = vfma(tx, vcx, vfma(vsub(fy_b, fy_t), vcy, vmul(vsub(zb[r], fz), vcz)));
        zb[r] = fz;
        fy_b = fy_t;
        if (CP == 2 && KL_ZBC == 1 && k == 0) t = vsplat(C(0));
        const int j = ty0 + yr;
        if (j < (int)a.ny) {
            const long long o = (long long)c0 + (long long)j * a.sj + (long long)k * a.sk;
            if (c0 + 1 < (int)a.nx) {
#if KL_ACC
                t = vadd(t, vldo(dst + o));
#endif
                vsto(dst + o, t);
            } else if (c0 < (int)a.nx) {
                outg(dst + o, vlo(t));
            }
        }
    }
}
#undef KL_P
#endif  // KL_CS

// ---- periodic x inside the kernel.  On a grid with nx >= 64 + H, the one
// tile whose reach [tx0 - H, tx0 + 64 + H) crosses x = 0 (or x = nx) loads,
// with each plane, a strip of 32 bytes x KL_ROWS rows per field that holds the
// interior columns its halo wraps to; once the plane has landed each thread
// copies its share of those values over the halo columns (between its wait
// and the level's barrier).  The kernel then reads no x ghost column of
// memory: the y and z ghosts must be filled, the x ghosts of interior rows
// need not be.  Narrower grids read the filled x ghosts.
#define KL_XW_W (32 / (int)sizeof(T))                        // strip width, elements
#define KL_STRIP_BOX (KL_ROWS * 32)                          // bytes one strip box lands
#define KL_STRIP_BYTES KL_RUP(KL_STRIP_BOX, 128)
#if KL_DIFF == 2
// variable nu: no x-wrap strips (the x ghosts are read from memory); nu ring
#define KL_ZSLOT (3 * KL_PLANE_BYTES)                        // zpack ring slot
#define KL_NROWS (KL_TYS + 2)                                // nu box: tile rows -1 .. TYS
#define KL_NBOX (KL_PITCH * KL_NROWS * (int)sizeof(T))
#define KL_NPLANE KL_RUP(KL_NBOX, 128)
#define KL_NLEAD (KL_R - 1)                                  // nu plane p - NLEAD rides with plane p
#else
#define KL_ZSLOT (3 * KL_PLANE_BYTES + 3 * KL_STRIP_BYTES)   // zpack ring slot
#endif
// carry mode: with one warp group, a ring of fewer than 2R+2 slots holds
// planes k-1 .. k+R plus one in flight; the own-column values of plane k-2
// that the vertical windows still need were read at the level before and
// stay in registers.  The first level's bottom faces, which reach down to
// plane kb-R, are formed before the level loop while planes kb-R .. kb+R-1
// fill the ring.  (Variable nu reads plane k-1 and above only.)
#define KL_CARRY (KL_NS < 2 * KL_R + 2)
#if KL_CARRY && (KL_CS || KL_NS < 2 * KL_R || KL_R < 2)
#error "a ring of fewer than 2R+2 slots needs cs=0, R >= 2 and at least 2R slots"
#endif
#if KL_DIFF == 2
// nu ring slots: planes k-1 .. k+1 plus one per u, v, w plane in flight
// (nu plane q rides with plane q + NLEAD): the ring holds planes k-R .. k+R,
// or k-1 .. k+R in carry mode, and the rest of its slots are in flight
#define KL_NNS (KL_CARRY ? KL_NS - KL_R + 1 : KL_NS - 2 * KL_R + 2)
#endif
#define KL_NT (32 * KL_MBY * (KL_CS ? 3 : 1))                // threads per block
#define KL_XW_Q ((3 * KL_ROWS * KL_H + KL_NT - 1) / KL_NT)   // halo values per thread
static_assert(KL_AL - 1 + KL_H - 1 < KL_XW_W, "a strip must hold the wrapped columns");

#if KL_DIFF == 2
#define KL_NOFF(x, row) ((((row) + 1) * KL_PITCH + (x)) * (int)sizeof(T))
// aligned pair of nu on plane k+DK at columns (lx + DX, lx + DX + 1), tile row
// `row` in [-1, TYS]
template <int DK, int DX>
__device__ __forceinline__ V kl_npr(const char *const *npl, int lx, int row)
{
    static_assert(DK >= -1 && DK <= 1, "nu plane outside the staged window");
    static_assert(DX % 2 == 0 && DX >= -KL_LPAD && KL_LPAD + 62 + DX + 1 < KL_PITCH, "nu x offset");
    return vld((const T *)(npl[DK + 1] + KL_NOFF(lx + DX, row)));
}
#endif

#if KL_YX == 2
// bottom y face of field F at tile row yr, on the level whose ring planes are
// P (P[R] the level's plane, P[R-1] the one below): the expressions of the
// row loop
template <int F>
__device__ __forceinline__ V kl_yface(const kl_vk &K, const char *const *P, int lx, int yr, V kd)
{
#define KL_P2(f, dk, dx, row) kl_pr<(f), (dk), (dx)>(P, lx, (row))
    V us;
    if constexpr (F == 0) us = vadd(vcross(KL_P2(1, 0, -2, yr), KL_P2(1, 0, 0, yr)), KL_P2(1, 0, 0, yr));
    else if constexpr (F == 1) us = vadd(KL_P2(1, 0, 0, yr - 1), KL_P2(1, 0, 0, yr));
    else us = vadd(KL_P2(1, -1, 0, yr), KL_P2(1, 0, 0, yr));
    return kl_vflux(K, us, KL_A5(KL_P2(F, 0, 0, yr - 3)), KL_A5(KL_P2(F, 0, 0, yr - 2)),
                    KL_P2(F, 0, 0, yr - 1), KL_P2(F, 0, 0, yr), KL_A5(KL_P2(F, 0, 0, yr + 1)),
                    KL_A5(KL_P2(F, 0, 0, yr + 2)), kd);
#undef KL_P2
}

// x face of field f beyond the tile's 64 columns at tile row `row` (u: the
// face at centre x0-1; v, w: the face at edge x0+64), scalar, as the side
// pass forms it
__device__ __forceinline__ C kl_xside(const char *const *P, int f, int row, C kdx)
{
    const int xs = f == 0 ? KL_LPAD - 3 : KL_LPAD + 61;
    const char *base = P[KL_R] + f * KL_PLANE_BYTES;
    C a2 = lds((const T *)(base + KL_OFF(xs + 2, row)));
    C a3 = lds((const T *)(base + KL_OFF(xs + 3, row)));
#if KL_ADV == 5
    C a0 = lds((const T *)(base + KL_OFF(xs, row)));
    C a1 = lds((const T *)(base + KL_OFF(xs + 1, row)));
    C a4 = lds((const T *)(base + KL_OFF(xs + 4, row)));
    C a5 = lds((const T *)(base + KL_OFF(xs + 5, row)));
#else
    C a0 = C(0), a1 = C(0), a4 = C(0), a5 = C(0);
#endif
    const char *p1 = f == 0 ? base + KL_OFF(xs + 2, row)
                   : (f == 1 ? P[KL_R] + KL_OFF(KL_LPAD + 64, row - 1)
                             : P[KL_R - 1] + KL_OFF(KL_LPAD + 64, row));
    const char *p2 = f == 0 ? base + KL_OFF(xs + 3, row) : P[KL_R] + KL_OFF(KL_LPAD + 64, row);
    const C us = lds((const T *)p1) + lds((const T *)p2);
    return kl_sflux(us, a0, a1, a2, a3, a4, a5, kdx);
}
#endif

// One tile (bxi, byi) over levels [kb, ke): the ring's prologue, then the
// level loop.  reinit: the ring's mbarriers were used by an earlier segment
// of the same CTA (all of their copies completed); they are invalidated and
// initialised again.  Returns false when a device wait gave up.
__device__ __forceinline__ bool kl_zpack_body(const kl_args &a, const kl_tmap *const *maps,
                                              int bxi, int byi, int kb, int ke, bool reinit)
{
    static_assert(KL_MBX == 32 && KL_MPX == 2, "zpack tiles are 64 columns wide");
    static_assert(3 * KL_MPY <= 32, "side pass needs 3 x rows <= 32 lanes");
    // reach of the pairs and the side pass: 4 columns left and right of the
    // tile for the 5th-order scheme, 2 left and 1 right otherwise
    static_assert(KL_LPAD % 2 == 0 && KL_LPAD >= (KL_ADV == 5 ? 4 : 2), "left pad too small");
    static_assert(KL_PITCH >= KL_LPAD + 64 + (KL_ADV == 5 ? 3 : 1), "right pad too small");
    extern __shared__ unsigned char kl_smem_raw[];
    // 128-byte aligned ring start, formed by pointer arithmetic on the shared
    // array so that every access below stays a shared-memory access (an
    // integer round trip would turn them into generic loads)
    unsigned char *ring = kl_smem_raw + ((128u - (kl_smem_addr(kl_smem_raw) & 127u)) & 127u);
#if KL_DIFF == 2
    unsigned char *nring = ring + KL_NS * KL_ZSLOT;
    unsigned long long *bars = (unsigned long long *)(nring + KL_NNS * KL_NPLANE);
#else
    unsigned long long *bars = (unsigned long long *)(ring + KL_NS * KL_ZSLOT);
#endif
#if KL_YX == 1
    // y-face exchange buffer after the barriers: [3 fields][warps][32 lanes]
    V *xbuf = (V *)((unsigned char *)bars + KL_RUP(8 * KL_NS, 16));
#elif KL_YX == 2
    // one level ahead, by level parity: the bottom y faces of each warp's
    // first row [2][3][warps][32 lanes], the tile's top y faces [2][3][32]
    // and the x faces beyond the tile's columns [2][3][TYS]
    V *ysh = (V *)((unsigned char *)bars + KL_RUP(8 * KL_NS, 16));
    V *ytop = ysh + 2 * 3 * KL_MBY * 32;
    C *sside = (C *)(ytop + 2 * 3 * 32);
#endif
    const int lane = threadIdx.x;
    const int warp = KL_CS ? (int)threadIdx.y % KL_MBY : (int)threadIdx.y;
    const int tid = lane + 32 * (int)threadIdx.y;
    const int nx = (int)a.nx, ny = (int)a.ny, nz = (int)a.nz;
    const int tx0 = bxi * 64, ty0 = byi * KL_TYS;
    const int gx = (int)a.tile_x0 + tx0 - KL_LPAD, gy = (int)a.tile_y0 + ty0 - KL_H;
    const int gz0 = (int)a.tile_z0;

    if (tid == 0) {
        if (reinit)
            for (int s = 0; s < KL_NS; ++s)
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(kl_smem_addr(&bars[s])) : "memory");
        for (int s = 0; s < KL_NS; ++s) kl_mbar_init(kl_smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // x wrap (see above): which side this tile wraps, never both
    const bool xw_on = KL_DIFF != 2 && nx >= 64 + KL_H && !(a.flags & 1);
    const bool need_l = xw_on && tx0 == 0, need_r = xw_on && tx0 + 64 + KL_H > nx;
    const bool xwrap = need_l || need_r;
    const int xs0 = need_l ? (nx - KL_H) / KL_AL * KL_AL : 0;   // first strip column
    auto issue = [&](int p) {
        int slot = (p - (kb - KL_R)) % KL_NS;
        unsigned bar = kl_smem_addr(&bars[slot]);
#if KL_DIFF == 2
        // nu plane q rides with plane p; planes below kb - 1 are never read
        const int q = p - KL_NLEAD;
        kl_mbar_expect(bar, 3 * KL_BOX_BYTES + (q >= kb - 1 ? KL_NBOX : 0));
#else
        kl_mbar_expect(bar, 3 * KL_BOX_BYTES + (xwrap ? 3 * KL_STRIP_BOX : 0));
#endif
        unsigned dst = kl_smem_addr(ring + slot * KL_ZSLOT);
#pragma unroll
        for (int f = 0; f < 3; ++f)
            kl_tma_load3(dst + f * KL_PLANE_BYTES, maps[f], gx, gy, gz0 + p, bar);
#if KL_DIFF == 2
        if (q >= kb - 1)
            kl_tma_load3(kl_smem_addr(nring + ((q - (kb - 1)) % KL_NNS) * KL_NPLANE), maps[3], gx,
                         (int)a.tile_y0 + ty0 - 1, gz0 + q, bar);
#endif
        if (xwrap) {
            // the halo columns of this slot were last written through the
            // generic proxy; order that before the asynchronous writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
            for (int f = 0; f < 3; ++f)
                kl_tma_load3(dst + 3 * KL_PLANE_BYTES + f * KL_STRIP_BYTES, maps[4 + f],
                             (int)a.tile_x0 + xs0, gy, gz0 + p, bar);
        }
    };
    const int p_first = kb - KL_R;
    const int p_last = ke - 1 + KL_R;
    int p_next = p_first;
    if (tid == 0)
        for (; p_next < p_first + KL_NS && p_next <= p_last; ++p_next) issue(p_next);
    // this thread's share of the halo values: byte offsets in a slot of the
    // strip source and the halo destination (-1: none)
    int xw_src[KL_XW_Q], xw_dst[KL_XW_Q];
#pragma unroll
    for (int t = 0; t < KL_XW_Q; ++t) {
        const int q = tid + t * KL_NT;
        const int f = q / (KL_ROWS * KL_H), rr = (q / KL_H) % KL_ROWS, c = q % KL_H;
        const int col = need_l ? nx - KL_H + c : c;             // wrapped-to column
        const bool ok = xwrap && q < 3 * KL_ROWS * KL_H && !(need_r && nx - tx0 + c >= 64 + KL_H);
        const int lc = need_l ? KL_LPAD - KL_H + c : KL_LPAD + (nx - tx0) + c;
        xw_src[t] = ok ? 3 * KL_PLANE_BYTES + f * KL_STRIP_BYTES + (rr * KL_XW_W + col - xs0) * (int)sizeof(T) : -1;
        xw_dst[t] = ok ? f * KL_PLANE_BYTES + (rr * KL_PITCH + lc) * (int)sizeof(T) : -1;
    }
    auto xw_copy = [&](unsigned char *slot) {
#pragma unroll
        for (int t = 0; t < KL_XW_Q; ++t)
            if (xw_src[t] >= 0) *(T *)(slot + xw_dst[t]) = *(const T *)(slot + xw_src[t]);
    };
    auto slot_of = [&](int p) { return ring + ((unsigned)(p - p_first) % KL_NS) * KL_ZSLOT; };

    // coefficients (f32 kernels read the f32 copies; no f64 arithmetic)
    const C dxi = KL_CO(a, 0), dyi = KL_CO(a, 1), nu = KL_CO(a, 4);
    const C kdx = nu * dxi / KL_FS;
    kl_vk K;
    K.c37 = vsplat(C(37)); K.cm8 = vsplat(C(-8)); K.c10 = vsplat(C(10)); K.cm5 = vsplat(C(-5));
    K.cm10 = vsplat(C(-10)); K.c5 = vsplat(C(5));
    const V vkdx = vsplat(kdx), vkdy = vsplat(nu * dyi / KL_FS);
    const V vcx = vsplat(KL_FS * dxi), vcy = vsplat(KL_FS * dyi);

    const int r0 = warp * KL_MPY;                       // first row of this thread (tile local)
    const int lx = KL_LPAD + 2 * lane;                  // local x of column c0 (even)
    const int c0 = tx0 + 2 * lane;                      // global interior column of c0
#if KL_YX == 2
    static_assert(KL_CARRY && KL_DIFF != 2 && !KL_CS, "yx=2 needs the carried ring and constant nu");
    // the next level's shared values, formed from its planes P: this warp's
    // first-row bottom y faces (kept in fyb0 and published for the warp
    // below), and, spread over the warps, the tile's x side faces and its
    // top y faces, all by level parity
    V fyb0[3];
    auto publish = [&](const char *const *P, int par) {
        fyb0[0] = kl_yface<0>(K, P, lx, r0, vkdy);
        fyb0[1] = kl_yface<1>(K, P, lx, r0, vkdy);
        fyb0[2] = kl_yface<2>(K, P, lx, r0, vkdy);
#pragma unroll
        for (int f = 0; f < 3; ++f) ysh[((par * 3 + f) * KL_MBY + warp) * 32 + lane] = fyb0[f];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            if (warp == f % KL_MBY)
                for (int row = lane; row < KL_TYS; row += 32)
                    sside[(par * 3 + f) * KL_TYS + row] = kl_xside(P, f, row, kdx);
        }
        if (warp == (KL_MBY - 1) % KL_MBY) ytop[(par * 3 + 0) * 32 + lane] = kl_yface<0>(K, P, lx, KL_TYS, vkdy);
        if (warp == (KL_MBY + KL_MBY - 2) % KL_MBY) ytop[(par * 3 + 1) * 32 + lane] = kl_yface<1>(K, P, lx, KL_TYS, vkdy);
        if (warp == (KL_MBY + KL_MBY - 3) % KL_MBY) ytop[(par * 3 + 2) * 32 + lane] = kl_yface<2>(K, P, lx, KL_TYS, vkdy);
    };
#endif

#if KL_CS
    const int grp = (int)threadIdx.y / KL_MBY;           // tendency component of this warp
    V zb[KL_MPY];
#else
    V zb[KL_MPY][3];
#endif
#if KL_DIFF == 2
    V sxz[KL_MPY], syz[KL_MPY];     // stresses of the xz and yz edges at zh_k, per row
#endif
    bool timed_out = false;
    int p_waited = p_first - 1;

    // planes of the first level; afterwards each level ends with the wait for
    // the next level's newest plane and one barrier that both releases the
    // slot of plane k-R and makes the time-out decision uniform
#if KL_CARRY
    V zc[KL_MPY][3];    // own values of plane k-2 (u, v, w) per row
#endif
    {
        bool ok = true;
        const int q_last = KL_CARRY ? kb + KL_R - 1 : kb + KL_R;
        for (int q = p_first; q <= q_last && ok; ++q) {
            ok = kl_mbar_wait(kl_smem_addr(&bars[(q - p_first) % KL_NS]), ((q - p_first) / KL_NS) & 1,
                              a.wait_cycles);
            if (ok && xwrap) xw_copy(slot_of(q));
        }
        timed_out = __syncthreads_or(!ok);
        if (!timed_out) p_waited = q_last;
    }
#if KL_CARRY
    if (!timed_out) {
        // bottom faces of level kb (planes kb-R .. kb+R-1) and the carried
        // plane kb-2; then the slots of kb-R and kb-R+1 take the next planes
        // and the first level waits for plane kb+R
        const char *pl[2 * KL_R + 1];
#pragma unroll
        for (int d = -KL_R; d <= KL_R; ++d)        // d = R: not landed yet, never read here
            pl[d + KL_R] = (const char *)(ring + ((unsigned)(kb + d - p_first) % KL_NS) * KL_ZSLOT);
        const kl_zmetric Z = kl_make_z(a, kb);
        const V kzu_b = vsplat(nu * Z.dzhi / KL_FS), kzw_b = vsplat(nu * Z.dzi_dn / KL_FS);
#pragma unroll
        for (int r = 0; r < KL_MPY; ++r) {
            const int yr = r0 + r;
            const V u_0 = kl_pr<0, 0, 0>(pl, lx, yr), v_0 = kl_pr<1, 0, 0>(pl, lx, yr),
                    w_0 = kl_pr<2, 0, 0>(pl, lx, yr);
            zb[r][0] = kl_vflux(K, vadd(vcross(kl_pr<2, 0, -2>(pl, lx, yr), w_0), w_0),
                                kl_pr<0, -3, 0>(pl, lx, yr), kl_pr<0, -2, 0>(pl, lx, yr),
                                kl_pr<0, -1, 0>(pl, lx, yr), u_0, kl_pr<0, 1, 0>(pl, lx, yr),
                                kl_pr<0, 2, 0>(pl, lx, yr), kzu_b);
            zb[r][1] = kl_vflux(K, vadd(kl_pr<2, 0, 0>(pl, lx, yr - 1), w_0),
                                kl_pr<1, -3, 0>(pl, lx, yr), kl_pr<1, -2, 0>(pl, lx, yr),
                                kl_pr<1, -1, 0>(pl, lx, yr), v_0, kl_pr<1, 1, 0>(pl, lx, yr),
                                kl_pr<1, 2, 0>(pl, lx, yr), kzu_b);
            zb[r][2] = kl_vflux(K, vadd(kl_pr<2, -1, 0>(pl, lx, yr), w_0),
                                kl_pr<2, -3, 0>(pl, lx, yr), kl_pr<2, -2, 0>(pl, lx, yr),
                                kl_pr<2, -1, 0>(pl, lx, yr), w_0, kl_pr<2, 1, 0>(pl, lx, yr),
                                kl_pr<2, 2, 0>(pl, lx, yr), kzw_b);
            zc[r][0] = kl_pr<0, -2, 0>(pl, lx, yr);
            zc[r][1] = kl_pr<1, -2, 0>(pl, lx, yr);
            zc[r][2] = kl_pr<2, -2, 0>(pl, lx, yr);
        }
#if KL_YX == 2
        publish(pl, kb & 1);
#endif
        __syncthreads();                            // planes kb-R, kb-R+1 read for the last time
        if (tid == 0)
            for (int t = 0; t < 2 && p_next <= p_last; ++t) issue(p_next++);
        bool ok = true;
        {
            const int q = kb + KL_R;
            ok = kl_mbar_wait(kl_smem_addr(&bars[(q - p_first) % KL_NS]), ((q - p_first) / KL_NS) & 1,
                              a.wait_cycles);
            if (ok && xwrap) xw_copy(slot_of(q));
        }
        timed_out = __syncthreads_or(!ok);
        if (!timed_out) p_waited = kb + KL_R;
    }
#endif
    for (int k = kb; k < ke && !timed_out; ++k) {
        const char *pl[2 * KL_R + 1];
#pragma unroll
        for (int d = -KL_R; d <= KL_R; ++d)
            pl[d + KL_R] = (const char *)(ring + ((unsigned)(k + d - p_first) % KL_NS) * KL_ZSLOT);
#define KL_Q(f, dk, dx, row) kl_pr<f, dk, dx>(pl, lx, row)

        const kl_zmetric Z = kl_make_z(a, k);
#if KL_CS
        if (grp == 0)
            kl_cs_level<0>(a, K, pl, Z, lane, lx, r0, c0, ty0, k, kb, nu, kdx, vkdx, vkdy, vcx, vcy, zb);
        else if (grp == 1)
            kl_cs_level<1>(a, K, pl, Z, lane, lx, r0, c0, ty0, k, kb, nu, kdx, vkdx, vkdy, vcx, vcy, zb);
        else
            kl_cs_level<2>(a, K, pl, Z, lane, lx, r0, c0, ty0, k, kb, nu, kdx, vkdx, vkdy, vcx, vcy, zb);
#else
        const V vczu = vsplat(KL_FS * Z.dzi), vczw = vsplat(KL_FS * Z.dzhi);
        const V vkzu_top = vsplat(nu * Z.dzhi_up / KL_FS);   // u, v top face zh_{k+1}
        const V vkzw_top = vsplat(nu * Z.dzi / KL_FS);       // w top face z_k
#if KL_DIFF == 2
        // nu planes k-1 .. k+1 and the stress coefficients of this level
        const char *npl[3];
#pragma unroll
        for (int d = -1; d <= 1; ++d)
            npl[d + 1] = (const char *)(nring + ((unsigned)(k + d - (kb - 1)) % KL_NNS) * KL_NPLANE);
#define KL_N(dk, dx, row) kl_npr<(dk), (dx)>(npl, lx, (row))
        // nu summed over the two columns (c-1, c) of an xh edge
#define KL_NSX(dk, row) vadd(vcross(KL_N(dk, -2, row), KL_N(dk, 0, row)), KL_N(dk, 0, row))
        const V kxn = vsplat(C(2) * dxi / KL_FS), kyn = vsplat(C(2) * dyi / KL_FS);
        const V kzn = vsplat(C(2) * Z.dzi / KL_FS);
        const V kx4 = vsplat(dxi / (C(4) * KL_FS)), ky4 = vsplat(dyi / (C(4) * KL_FS));
        const V kz4t = vsplat(Z.dzhi_up / (C(4) * KL_FS)), kz4b = vsplat(Z.dzhi / (C(4) * KL_FS));
        // the term an edge stress adds to a face flux, -S / FS, with S =
        // (nu4 / 4) (difference along the face normal x metric + cross
        // difference x metric): d1 = a_m - a_{m+1} of the face's own window
        auto shear = [&](V nu4, V d1, V ka, V db, V kb_) {
            return vmul(nu4, vsub(vmul(d1, ka), vmul(db, kb_)));
        };
        if (k == kb) {
            // z-edge stresses at zh_k of the first level (carried afterwards)
#pragma unroll
            for (int r = 0; r < KL_MPY; ++r) {
                const int yr = r0 + r;
                const V u_0 = KL_Q(0, 0, 0, yr), w_0 = KL_Q(2, 0, 0, yr);
                sxz[r] = shear(vadd(KL_NSX(-1, yr), KL_NSX(0, yr)), vsub(KL_Q(0, -1, 0, yr), u_0), kz4b,
                               vsub(w_0, vcross(KL_Q(2, 0, -2, yr), w_0)), kx4);
                syz[r] = shear(vadd(vadd(KL_N(-1, 0, yr - 1), KL_N(-1, 0, yr)),
                                    vadd(KL_N(0, 0, yr - 1), KL_N(0, 0, yr))),
                               vsub(KL_Q(1, -1, 0, yr), KL_Q(1, 0, 0, yr)), kz4b,
                               vsub(w_0, KL_Q(2, 0, 0, yr - 1)), ky4);
            }
        }
#endif

        // ---- side pass: the x face beyond the warp's columns, every row
#if KL_YX != 2
        C extra;
        {
            int e = lane < 3 * KL_MPY ? lane : 0;
            int f = e / KL_MPY, row = r0 + e % KL_MPY;
            // u: face at centre x0-1 (values x0-3 .. x0+2, Us = a2 + a3);
            // v, w: face at edge x0+64 (values x0+61 .. x0+66, Us = two u's)
            int xs = f == 0 ? KL_LPAD - 3 : KL_LPAD + 61;
            const char *base = pl[KL_R] + f * KL_PLANE_BYTES;
            C a2 = lds((const T *)(base + KL_OFF(xs + 2, row)));
            C a3 = lds((const T *)(base + KL_OFF(xs + 3, row)));
#if KL_ADV == 5
            C a0 = lds((const T *)(base + KL_OFF(xs, row)));
            C a1 = lds((const T *)(base + KL_OFF(xs + 1, row)));
            C a4 = lds((const T *)(base + KL_OFF(xs + 4, row)));
            C a5 = lds((const T *)(base + KL_OFF(xs + 5, row)));
#else
            C a0 = C(0), a1 = C(0), a4 = C(0), a5 = C(0);
#endif
            // branch-free choice of the two velocities that form Us
            const char *p1 = f == 0 ? base + KL_OFF(xs + 2, row)
                           : (f == 1 ? pl[KL_R] + KL_OFF(KL_LPAD + 64, row - 1)
                                     : pl[KL_R - 1] + KL_OFF(KL_LPAD + 64, row));
            const char *p2 = f == 0 ? base + KL_OFF(xs + 3, row) : pl[KL_R] + KL_OFF(KL_LPAD + 64, row);
            C us = lds((const T *)p1) + lds((const T *)p2);
            extra = kl_sflux(us, a0, a1, a2, a3, a4, a5, kdx);
#if KL_DIFF == 2
            {
                // the face's stress, as the pair code forms it
                const C nl = lds((const T *)(npl[1] + KL_NOFF(KL_LPAD + 63, row)));
                const C nr = lds((const T *)(npl[1] + KL_NOFF(KL_LPAD + 64, row)));
                const C d1c = lds((const T *)p1) - lds((const T *)p2);   // cross: two u's
                C st;
                if (f == 0) {
                    st = C(2) * dxi / KL_FS * lds((const T *)(npl[1] + KL_NOFF(KL_LPAD - 1, row))) * (a2 - a3);
                } else if (f == 1) {
                    const C nu4 = lds((const T *)(npl[1] + KL_NOFF(KL_LPAD + 63, row - 1))) +
                                  lds((const T *)(npl[1] + KL_NOFF(KL_LPAD + 64, row - 1))) + nl + nr;
                    st = nu4 * (d1c * (dyi / (C(4) * KL_FS)) - (a3 - a2) * (dxi / (C(4) * KL_FS)));
                } else {
                    const C nu4 = lds((const T *)(npl[0] + KL_NOFF(KL_LPAD + 63, row))) +
                                  lds((const T *)(npl[0] + KL_NOFF(KL_LPAD + 64, row))) + nl + nr;
                    st = nu4 * (d1c * (Z.dzhi / (C(4) * KL_FS)) - (a3 - a2) * (dxi / (C(4) * KL_FS)));
                }
                extra += st;
            }
#endif
        }
#endif

        // ---- y faces
#if KL_YX == 1
        // every thread forms the bottom faces of its rows; the top face of
        // its last row is the bottom face of the warp above, exchanged
        // through shared memory (the last warp forms the tile's top face)
        V fyb[KL_MPY][3], fyt_last[3];
#pragma unroll
        for (int r = 0; r < KL_MPY; ++r) {
            const int yr = r0 + r;
            fyb[r][0] = kl_vflux(K, vadd(vcross(KL_Q(1, 0, -2, yr), KL_Q(1, 0, 0, yr)), KL_Q(1, 0, 0, yr)),
                                 KL_A5(KL_Q(0, 0, 0, yr - 3)), KL_A5(KL_Q(0, 0, 0, yr - 2)), KL_Q(0, 0, 0, yr - 1),
                                 KL_Q(0, 0, 0, yr), KL_A5(KL_Q(0, 0, 0, yr + 1)), KL_A5(KL_Q(0, 0, 0, yr + 2)), vkdy);
            fyb[r][1] = kl_vflux(K, vadd(KL_Q(1, 0, 0, yr - 1), KL_Q(1, 0, 0, yr)),
                                 KL_A5(KL_Q(1, 0, 0, yr - 3)), KL_A5(KL_Q(1, 0, 0, yr - 2)), KL_Q(1, 0, 0, yr - 1),
                                 KL_Q(1, 0, 0, yr), KL_A5(KL_Q(1, 0, 0, yr + 1)), KL_A5(KL_Q(1, 0, 0, yr + 2)), vkdy);
            fyb[r][2] = kl_vflux(K, vadd(KL_Q(1, -1, 0, yr), KL_Q(1, 0, 0, yr)),
                                 KL_A5(KL_Q(2, 0, 0, yr - 3)), KL_A5(KL_Q(2, 0, 0, yr - 2)), KL_Q(2, 0, 0, yr - 1),
                                 KL_Q(2, 0, 0, yr), KL_A5(KL_Q(2, 0, 0, yr + 1)), KL_A5(KL_Q(2, 0, 0, yr + 2)), vkdy);
        }
#pragma unroll
        for (int f = 0; f < 3; ++f) xbuf[(f * KL_MBY + warp) * 32 + lane] = fyb[0][f];
        if (warp == KL_MBY - 1) {
            const int yt = r0 + KL_MPY;
            fyt_last[0] = kl_vflux(K, vadd(vcross(KL_Q(1, 0, -2, yt), KL_Q(1, 0, 0, yt)), KL_Q(1, 0, 0, yt)),
                                   KL_A5(KL_Q(0, 0, 0, yt - 3)), KL_A5(KL_Q(0, 0, 0, yt - 2)), KL_Q(0, 0, 0, yt - 1),
                                   KL_Q(0, 0, 0, yt), KL_A5(KL_Q(0, 0, 0, yt + 1)), KL_A5(KL_Q(0, 0, 0, yt + 2)), vkdy);
            fyt_last[1] = kl_vflux(K, vadd(KL_Q(1, 0, 0, yt - 1), KL_Q(1, 0, 0, yt)),
                                   KL_A5(KL_Q(1, 0, 0, yt - 3)), KL_A5(KL_Q(1, 0, 0, yt - 2)), KL_Q(1, 0, 0, yt - 1),
                                   KL_Q(1, 0, 0, yt), KL_A5(KL_Q(1, 0, 0, yt + 1)), KL_A5(KL_Q(1, 0, 0, yt + 2)), vkdy);
            fyt_last[2] = kl_vflux(K, vadd(KL_Q(1, -1, 0, yt), KL_Q(1, 0, 0, yt)),
                                   KL_A5(KL_Q(2, 0, 0, yt - 3)), KL_A5(KL_Q(2, 0, 0, yt - 2)), KL_Q(2, 0, 0, yt - 1),
                                   KL_Q(2, 0, 0, yt), KL_A5(KL_Q(2, 0, 0, yt + 1)), KL_A5(KL_Q(2, 0, 0, yt + 2)), vkdy);
        } else {
            fyt_last[0] = fyt_last[1] = fyt_last[2] = vsplat(C(0));
        }
        __syncthreads();
        if (warp != KL_MBY - 1) {
#pragma unroll
            for (int f = 0; f < 3; ++f) fyt_last[f] = xbuf[(f * KL_MBY + warp + 1) * 32 + lane];
        }
        V fuy_b = fyb[0][0], fvy_b = fyb[0][1], fwy_b = fyb[0][2];
#elif KL_YX == 2
        const int par = k & 1;
        V fuy_b = fyb0[0], fvy_b = fyb0[1], fwy_b = fyb0[2];
#else
        V fuy_b, fvy_b, fwy_b;
        {
            const int yr = r0;
            fuy_b = kl_vflux(K, vadd(vcross(KL_Q(1, 0, -2, yr), KL_Q(1, 0, 0, yr)), KL_Q(1, 0, 0, yr)),
                             KL_A5(KL_Q(0, 0, 0, yr - 3)), KL_A5(KL_Q(0, 0, 0, yr - 2)), KL_Q(0, 0, 0, yr - 1),
                             KL_Q(0, 0, 0, yr), KL_A5(KL_Q(0, 0, 0, yr + 1)), KL_A5(KL_Q(0, 0, 0, yr + 2)), vkdy);
            fvy_b = kl_vflux(K, vadd(KL_Q(1, 0, 0, yr - 1), KL_Q(1, 0, 0, yr)),
                             KL_A5(KL_Q(1, 0, 0, yr - 3)), KL_A5(KL_Q(1, 0, 0, yr - 2)), KL_Q(1, 0, 0, yr - 1),
                             KL_Q(1, 0, 0, yr), KL_A5(KL_Q(1, 0, 0, yr + 1)), KL_A5(KL_Q(1, 0, 0, yr + 2)), vkdy);
            fwy_b = kl_vflux(K, vadd(KL_Q(1, -1, 0, yr), KL_Q(1, 0, 0, yr)),
                             KL_A5(KL_Q(2, 0, 0, yr - 3)), KL_A5(KL_Q(2, 0, 0, yr - 2)), KL_Q(2, 0, 0, yr - 1),
                             KL_Q(2, 0, 0, yr), KL_A5(KL_Q(2, 0, 0, yr + 1)), KL_A5(KL_Q(2, 0, 0, yr + 2)), vkdy);
        }
#endif
#if KL_DIFF == 2
        // stress of the xy edge at the bottom of the current row: u's y face
        // and v's x face of that row
        V sxy;
        {
            const int yr = r0;
            const V v0 = KL_Q(1, 0, 0, yr);
            sxy = shear(vadd(KL_NSX(0, yr - 1), KL_NSX(0, yr)), vsub(KL_Q(0, 0, 0, yr - 1), KL_Q(0, 0, 0, yr)),
                        ky4, vsub(v0, vcross(KL_Q(1, 0, -2, yr), v0)), kx4);
            fuy_b = vadd(fuy_b, sxy);
            fvy_b = vfma(vmul(kyn, KL_N(0, 0, yr - 1)), vsub(KL_Q(1, 0, 0, yr - 1), v0), fvy_b);
            fwy_b = vadd(fwy_b, syz[0]);
        }
#endif

#pragma unroll
        for (int r = 0; r < KL_MPY; ++r) {
            const int yr = r0 + r;
            // ---- x faces of both columns: u right faces (centres), v, w left
            // faces (edges); pairs at even offsets, odd offsets by vcross
            V u_m2 = KL_A5(KL_Q(0, 0, -2, yr)), u_0 = KL_Q(0, 0, 0, yr), u_2 = KL_Q(0, 0, 2, yr);
            V fux = kl_vflux(K, vadd(u_0, vcross(u_0, u_2)),
                             KL_A5(u_m2), KL_A5(vcross(u_m2, u_0)), u_0,
                             vcross(u_0, u_2), KL_A5(u_2), KL_A5(vcross(u_2, KL_Q(0, 0, 4, yr))), vkdx);
            V v_m4 = KL_A5(KL_Q(1, 0, -4, yr)), v_m2 = KL_Q(1, 0, -2, yr), v_0 = KL_Q(1, 0, 0, yr),
              v_2 = KL_Q(1, 0, 2, yr);
            V fvx = kl_vflux(K, vadd(KL_Q(0, 0, 0, yr - 1), u_0),
                             KL_A5(vcross(v_m4, v_m2)), KL_A5(v_m2), vcross(v_m2, v_0),
                             v_0, KL_A5(vcross(v_0, v_2)), KL_A5(v_2), vkdx);
            V w_m4 = KL_A5(KL_Q(2, 0, -4, yr)), w_m2 = KL_Q(2, 0, -2, yr), w_0 = KL_Q(2, 0, 0, yr),
              w_2 = KL_Q(2, 0, 2, yr);
            V fwx = kl_vflux(K, vadd(KL_Q(0, -1, 0, yr), u_0),
                             KL_A5(vcross(w_m4, w_m2)), KL_A5(w_m2), vcross(w_m2, w_0),
                             w_0, KL_A5(vcross(w_0, w_2)), KL_A5(w_2), vkdx);
#if KL_DIFF == 2
            fux = vfma(vmul(kxn, KL_N(0, 0, yr)), vsub(u_0, vcross(u_0, u_2)), fux);
            fvx = vadd(fvx, sxy);
            fwx = vadd(fwx, sxz[r]);
#endif
            // faces on the other side: u left = (lane-1 hi, own lo);
            // v, w right = (own hi, lane+1 lo); warp edges from the side pass
            C ul_hi = __shfl_sync(0xffffffffu, vhi(fux), (lane + 31) & 31);
            C vr_lo = __shfl_sync(0xffffffffu, vlo(fvx), (lane + 1) & 31);
            C wr_lo = __shfl_sync(0xffffffffu, vlo(fwx), (lane + 1) & 31);
#if KL_YX == 2
            const C eu = sside[(par * 3 + 0) * KL_TYS + yr], ev = sside[(par * 3 + 1) * KL_TYS + yr],
                    ew = sside[(par * 3 + 2) * KL_TYS + yr];
#else
            C eu = __shfl_sync(0xffffffffu, extra, r);
            C ev = __shfl_sync(0xffffffffu, extra, KL_MPY + r);
            C ew = __shfl_sync(0xffffffffu, extra, 2 * KL_MPY + r);
#endif
            V ul = vmk(lane == 0 ? eu : ul_hi, vlo(fux));
            V vr = vmk(vhi(fvx), lane == 31 ? ev : vr_lo);
            V wr = vmk(vhi(fwx), lane == 31 ? ew : wr_lo);

            // ---- top y faces of this row
#if KL_YX == 1
            V fuy_t, fvy_t, fwy_t;
            if (r + 1 < KL_MPY) {
                fuy_t = fyb[r + 1 < KL_MPY ? r + 1 : 0][0];
                fvy_t = fyb[r + 1 < KL_MPY ? r + 1 : 0][1];
                fwy_t = fyb[r + 1 < KL_MPY ? r + 1 : 0][2];
            } else {
                fuy_t = fyt_last[0];
                fvy_t = fyt_last[1];
                fwy_t = fyt_last[2];
            }
#else
            const int yt = yr + 1;
            V fuy_t, fvy_t, fwy_t;
            if (KL_YX != 2 || r + 1 < KL_MPY) {
                fuy_t = kl_vflux(K, vadd(vcross(KL_Q(1, 0, -2, yt), KL_Q(1, 0, 0, yt)), KL_Q(1, 0, 0, yt)),
                                 KL_A5(KL_Q(0, 0, 0, yt - 3)), KL_A5(KL_Q(0, 0, 0, yt - 2)), KL_Q(0, 0, 0, yt - 1),
                                 KL_Q(0, 0, 0, yt), KL_A5(KL_Q(0, 0, 0, yt + 1)), KL_A5(KL_Q(0, 0, 0, yt + 2)), vkdy);
                fvy_t = kl_vflux(K, vadd(KL_Q(1, 0, 0, yt - 1), KL_Q(1, 0, 0, yt)),
                                 KL_A5(KL_Q(1, 0, 0, yt - 3)), KL_A5(KL_Q(1, 0, 0, yt - 2)), KL_Q(1, 0, 0, yt - 1),
                                 KL_Q(1, 0, 0, yt), KL_A5(KL_Q(1, 0, 0, yt + 1)), KL_A5(KL_Q(1, 0, 0, yt + 2)), vkdy);
                fwy_t = kl_vflux(K, vadd(KL_Q(1, -1, 0, yt), KL_Q(1, 0, 0, yt)),
                                 KL_A5(KL_Q(2, 0, 0, yt - 3)), KL_A5(KL_Q(2, 0, 0, yt - 2)), KL_Q(2, 0, 0, yt - 1),
                                 KL_Q(2, 0, 0, yt), KL_A5(KL_Q(2, 0, 0, yt + 1)), KL_A5(KL_Q(2, 0, 0, yt + 2)), vkdy);
            } else {
#if KL_YX == 2
                // the first-row bottom faces of the warp above, or the tile's
                // top faces, formed one level earlier
                const V *src = warp + 1 < KL_MBY ? ysh + (par * 3 * KL_MBY + warp + 1) * 32 + lane
                                                 : ytop + par * 3 * 32 + lane;
                const int fs = warp + 1 < KL_MBY ? KL_MBY * 32 : 32;
                fuy_t = src[0];
                fvy_t = src[fs];
                fwy_t = src[2 * fs];
#endif
            }
#endif
#if KL_DIFF == 2
            V sxy_t;
            {
                const int yt = yr + 1;
                const V v0t = KL_Q(1, 0, 0, yt);
                sxy_t = shear(vadd(KL_NSX(0, yr), KL_NSX(0, yt)), vsub(KL_Q(0, 0, 0, yr), KL_Q(0, 0, 0, yt)),
                              ky4, vsub(v0t, vcross(KL_Q(1, 0, -2, yt), v0t)), kx4);
                fuy_t = vadd(fuy_t, sxy_t);
                fvy_t = vfma(vmul(kyn, KL_N(0, 0, yr)), vsub(KL_Q(1, 0, 0, yr), v0t), fvy_t);
                // yz edge at the bottom of row yt: carried for the thread's own
                // rows, formed here above its last row
                V syz_t;
                if (r + 1 < KL_MPY)
                    syz_t = syz[r + 1 < KL_MPY ? r + 1 : 0];
                else
                    syz_t = shear(vadd(vadd(KL_N(-1, 0, yr), KL_N(-1, 0, yt)), vadd(KL_N(0, 0, yr), KL_N(0, 0, yt))),
                                  vsub(KL_Q(1, -1, 0, yt), v0t), kz4b, vsub(KL_Q(2, 0, 0, yt), KL_Q(2, 0, 0, yr)), ky4);
                fwy_t = vadd(fwy_t, syz_t);
            }
#endif

            // ---- z faces: bottom carried, top formed here
#if KL_CARRY
#define KL_QM2(f) zc[r][f]
#else
#define KL_QM2(f) KL_Q(f, -2, 0, yr)
#endif
            V fz_u = kl_vflux(K, vadd(vcross(KL_Q(2, 1, -2, yr), KL_Q(2, 1, 0, yr)), KL_Q(2, 1, 0, yr)),
                              KL_A5(KL_QM2(0)), KL_A5(KL_Q(0, -1, 0, yr)), u_0,
                              KL_Q(0, 1, 0, yr), KL_A5(KL_Q(0, 2, 0, yr)), KL_A5(KL_Q(0, 3, 0, yr)), vkzu_top);
            V fz_v = kl_vflux(K, vadd(KL_Q(2, 1, 0, yr - 1), KL_Q(2, 1, 0, yr)),
                              KL_A5(KL_QM2(1)), KL_A5(KL_Q(1, -1, 0, yr)), v_0,
                              KL_Q(1, 1, 0, yr), KL_A5(KL_Q(1, 2, 0, yr)), KL_A5(KL_Q(1, 3, 0, yr)), vkzu_top);
            V fz_w = kl_vflux(K, vadd(w_0, KL_Q(2, 1, 0, yr)),
                              KL_A5(KL_QM2(2)), KL_A5(KL_Q(2, -1, 0, yr)), w_0,
                              KL_Q(2, 1, 0, yr), KL_A5(KL_Q(2, 2, 0, yr)), KL_A5(KL_Q(2, 3, 0, yr)), vkzw_top);
#if !KL_CARRY
            if (k == kb) {
                // bottom faces of the first level: u, v at zh_k, w at z_{k-1}
                const V kzu_b = vsplat(nu * Z.dzhi / KL_FS), kzw_b = vsplat(nu * Z.dzi_dn / KL_FS);
                zb[r][0] = kl_vflux(K, vadd(vcross(KL_Q(2, 0, -2, yr), w_0), w_0),
                                    KL_A5(KL_Q(0, -3, 0, yr)), KL_A5(KL_Q(0, -2, 0, yr)), KL_Q(0, -1, 0, yr),
                                    u_0, KL_A5(KL_Q(0, 1, 0, yr)), KL_A5(KL_Q(0, 2, 0, yr)), kzu_b);
                zb[r][1] = kl_vflux(K, vadd(KL_Q(2, 0, 0, yr - 1), w_0),
                                    KL_A5(KL_Q(1, -3, 0, yr)), KL_A5(KL_Q(1, -2, 0, yr)), KL_Q(1, -1, 0, yr),
                                    v_0, KL_A5(KL_Q(1, 1, 0, yr)), KL_A5(KL_Q(1, 2, 0, yr)), kzu_b);
                zb[r][2] = kl_vflux(K, vadd(KL_Q(2, -1, 0, yr), w_0),
                                    KL_A5(KL_Q(2, -3, 0, yr)), KL_A5(KL_Q(2, -2, 0, yr)), KL_Q(2, -1, 0, yr),
                                    w_0, KL_A5(KL_Q(2, 1, 0, yr)), KL_A5(KL_Q(2, 2, 0, yr)), kzw_b);
            }
#endif
#if KL_DIFF == 2
            {
                // top z faces: xz and yz edges at zh_{k+1}, w's normal stress at z_k
                const V w10 = KL_Q(2, 1, 0, yr);
                const V sxz_t = shear(vadd(KL_NSX(0, yr), KL_NSX(1, yr)), vsub(u_0, KL_Q(0, 1, 0, yr)), kz4t,
                                      vsub(w10, vcross(KL_Q(2, 1, -2, yr), w10)), kx4);
                const V syz_t = shear(vadd(vadd(KL_N(0, 0, yr - 1), KL_N(0, 0, yr)),
                                           vadd(KL_N(1, 0, yr - 1), KL_N(1, 0, yr))),
                                      vsub(v_0, KL_Q(1, 1, 0, yr)), kz4t, vsub(w10, KL_Q(2, 1, 0, yr - 1)), ky4);
                fz_u = vadd(fz_u, sxz_t);
                fz_v = vadd(fz_v, syz_t);
                fz_w = vfma(vmul(kzn, KL_N(0, 0, yr)), vsub(w_0, w10), fz_w);
                if (k == kb) {
                    zb[r][0] = vadd(zb[r][0], sxz[r]);
                    zb[r][1] = vadd(zb[r][1], syz[r]);
                    zb[r][2] = vfma(vmul(vsplat(C(2) * Z.dzi_dn / KL_FS), KL_N(-1, 0, yr)),
                                    vsub(KL_Q(2, -1, 0, yr), w_0), zb[r][2]);
                }
                sxz[r] = sxz_t;
                syz[r] = syz_t;
            }
#endif
            // ---- tendencies
            V tu = vfma(vsub(ul, fux), vcx, vfma(vsub(fuy_b, fuy_t), vcy, vmul(vsub(zb[r][0], fz_u), vczu)));
            V tv = vfma(vsub(fvx, vr), vcx, vfma(vsub(fvy_b, fvy_t), vcy, vmul(vsub(zb[r][1], fz_v), vczu)));
            V tw = vfma(vsub(fwx, wr), vcx, vfma(vsub(fwy_b, fwy_t), vcy, vmul(vsub(zb[r][2], fz_w), vczw)));
            zb[r][0] = fz_u;
            zb[r][1] = fz_v;
            zb[r][2] = fz_w;
#if KL_CARRY
            // plane k-1 is the next level's plane k-2
            zc[r][0] = KL_Q(0, -1, 0, yr);
            zc[r][1] = KL_Q(1, -1, 0, yr);
            zc[r][2] = KL_Q(2, -1, 0, yr);
#endif
#undef KL_QM2
            fuy_b = fuy_t;
            fvy_b = fvy_t;
            fwy_b = fwy_t;
#if KL_DIFF == 2
            sxy = sxy_t;
#endif
            if (KL_ZBC == 1 && k == 0) tw = vsplat(C(0));
            const int j = ty0 + yr;
            if (j < ny) {
                const long long o = (long long)c0 + (long long)j * a.sj + (long long)k * a.sk;
                if (c0 + 1 < nx) {
#if KL_ACC
                    tu = vadd(tu, vldo(a.ut + o));
                    tv = vadd(tv, vldo(a.vt + o));
                    tw = vadd(tw, vldo(a.wt + o));
#endif
                    vsto(a.ut + o, tu);
                    vsto(a.vt + o, tv);
                    vsto(a.wt + o, tw);
                } else if (c0 < nx) {
                    outg(a.ut + o, vlo(tu));
                    outg(a.vt + o, vlo(tv));
                    outg(a.wt + o, vlo(tw));
                }
            }
        }
#if KL_YX == 2
        if (k + 1 < ke) {
            // planes of level k+1: the ring's, shifted by one (its plane
            // k+1+R, still in flight, is never read here)
            const char *pln[2 * KL_R + 1];
#pragma unroll
            for (int d = 0; d < 2 * KL_R; ++d) pln[d] = pl[d + 1];
            pln[2 * KL_R] = pl[2 * KL_R];
            publish(pln, (k + 1) & 1);
        }
#endif
#if KL_DIFF == 2
#undef KL_N
#undef KL_NSX
#endif
#endif  // KL_CS
#undef KL_Q
        bool ok = true;
        if (k + 1 < ke) {
            const int p = k + 1 + KL_R;
            ok = kl_mbar_wait(kl_smem_addr(&bars[(p - p_first) % KL_NS]), ((p - p_first) / KL_NS) & 1,
                              a.wait_cycles);
            if (ok && xwrap) xw_copy(slot_of(p));
        }
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (k + 1 < ke) p_waited = k + 1 + KL_R;
        if (tid == 0 && p_next <= p_last) issue(p_next++);
    }

    if (timed_out) {
        if (tid == 0) {
            atomicOr(a.err, KL_DEV_TIMEOUT);
            for (int q = p_waited + 1; q < p_next; ++q) {
                unsigned b2 = kl_smem_addr(&bars[(q - p_first) % KL_NS]);
                kl_mbar_drain(b2, ((q - p_first) / KL_NS) & 1);
            }
        }
        __syncthreads();
    }
    return !timed_out;
}

#if KL_BATCH
extern "C" __global__ void __launch_bounds__(32 * KL_MBY * (KL_CS ? 3 : 1), KL_MMINB)
kl_tendency(const kl_args *argv, const int4 *blocks, const kl_tmap *tmaps)
{
    const int4 d = blocks[blockIdx.x];
    const kl_args a = argv[d.x];
    const kl_tmap *maps[7];
    for (int f = 0; f < 7; ++f) maps[f] = &tmaps[7 * d.x + f];
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int f = 0; f < 7; ++f) kl_tmap_acquire(maps[f]);
    const int kb = d.w * (int)a.kchunk;
    kl_zpack_body(a, maps, d.y, d.z, kb, min(kb + (int)a.kchunk, (int)a.nz), false);
}
#else
extern "C" __global__ void __launch_bounds__(32 * KL_MBY * (KL_CS ? 3 : 1), KL_MMINB)
kl_tendency(const kl_args a, const __grid_constant__ kl_tmap tm_u,
            const __grid_constant__ kl_tmap tm_v, const __grid_constant__ kl_tmap tm_w,
            const __grid_constant__ kl_tmap tm_n, const __grid_constant__ kl_tmap tm_su,
            const __grid_constant__ kl_tmap tm_sv, const __grid_constant__ kl_tmap tm_sw)
{
    // tm_su .. tm_sw: the same fields with the 32-byte x-wrap strip box
    const kl_tmap *maps[7] = {&tm_u, &tm_v, &tm_w, &tm_n, &tm_su, &tm_sv, &tm_sw};
#if KL_PE
    // Persistent CTAs.  A range [i, end) of a space of (tile, level) pairs,
    // tiles x fastest and each tile's levels lev0 .. lev0+nlev-1 consecutive,
    // runs as segments of consecutive levels of one tile: the plane ring's
    // prologue (and the re-read of the planes below a z chunk) happens once
    // per segment instead of once per chunk.
    bool first = true;
    auto run = [&](long long i, long long end, int nlev, int lev0) {
        while (i < end) {
            const long long t = i / nlev;
            const int k0 = (int)(i - t * nlev);
            const long long left = end - i;
            const int k1 = left < nlev - k0 ? k0 + (int)left : nlev;
            if (!first) __syncthreads();           // the last segment's ring is idle
            if (!kl_zpack_body(a, maps, (int)(t % a.nbx), (int)(t / a.nbx), lev0 + k0, lev0 + k1, !first))
                return false;
            first = false;
            i += k1 - k0;
        }
        return true;
    };
    const long long G = gridDim.x, ntile = a.nbx * a.nby, nz = a.nz;
    if (KL_PE == 2 && G > ntile) {
        // column-synchronous: CTA b < ntile marches tile b from level 0 to h,
        // so that these CTAs climb their columns together and a tile's halo
        // rows (its neighbours' rows of the same level) are read at about the
        // same time by both (the L2 keeps them); the other CTAs share the
        // levels h .. nz-1 of every tile in equal ranges.  h balances the two
        // kinds, counting about two levels of work for each ring prologue.
        const long long ne = G - ntile;
        const long long nseg = (ntile + ne - 1) / ne + 1;
        long long h = (ntile * nz + 2 * ne * (nseg - 1)) / G;
        h = h < 1 ? 1 : (h > nz ? nz : h);
        if ((long long)blockIdx.x < ntile) {
            run((long long)blockIdx.x * h, (long long)blockIdx.x * h + h, (int)h, 0);
        } else if (h < nz) {
            const long long tops = ntile * (nz - h), per = (tops + ne - 1) / ne;
            const long long i = ((long long)blockIdx.x - ntile) * per;
            run(i, i + per < tops ? i + per : tops, (int)(nz - h), (int)h);
        }
    } else {
        // equal contiguous ranges of all (tile, level) pairs: every CTA gets
        // the same number of levels (no partial last wave)
        const long long ntl = ntile * nz, per = (ntl + G - 1) / G;
        const long long i = (long long)blockIdx.x * per;
        run(i, ntl < i + per ? ntl : i + per, (int)nz, 0);
    }
#else
    const int kb = (int)blockIdx.z * (int)a.kchunk;
    kl_zpack_body(a, maps, blockIdx.x, blockIdx.y, kb, min(kb + (int)a.kchunk, (int)a.nz), false);
#endif
}
#endif
#endif  // KL_FAMILY == 2
