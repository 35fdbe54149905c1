/*
 * oracle.c -- plain, slow FP64 reference of the stencil tendencies.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * it is used by tests/, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg.  It shares no code, header or table with the CUDA path.
 *
 * What it computes.  The paper (Sec. 5.2) tunes two MicroHH kernels: advec_u,
 * the momentum-advection kernel whose face values use 5th-order
 * interpolation inside a 2nd-order scheme, and diff_uvw, the kernel of the
 * 2nd-order Smagorinsky diffusion.  It prints no formulas, so this file
 * writes out the standard staggered-grid (Arakawa C) flux-form finite
 * differences those names denote:
 *
 *   advection   tendency = -div(u_j u_i), face fluxes F = U * a_face, with the
 *               advecting velocity U averaged to the face (2nd order) and the
 *               advected a interpolated either by the 2-point mean (adv = 2),
 *               or by the 6-point upwind-biased 5th-order formula
 *               F5 = U*I6 + |U|*D6 (adv = 5, Wicker & Skamarock 2002),
 *               or by the centred 6th-order I6 alone (adv = 6; used only by
 *               the convergence-order tests);
 *   diffusion   diff = 1: nu * Laplacian with constant nu;
 *               diff = 2: stress divergence d_j[nu (d_j u_i + d_i u_j)] with a
 *               cell-centred eddy viscosity nu, 4-point averages of nu on
 *               cell edges;
 *   eddy viscosity  or_smagorinsky: nu = (cs delta)^2 sqrt(2 S_ij S_ij) of the
 *               Smagorinsky model, the nu that diff = 2 takes as input.
 *
 * Grid: interior i in [0,nx), j in [0,ny), k in [0,nz), g ghost cells on every
 * side.  u(i,j,k) sits at (i dx, (j+1/2) dy, z_k), v at ((i+1/2) dx, j dy, z_k),
 * w at ((i+1/2) dx, (j+1/2) dy, zh_k), nu at cell centres.  x and y are
 * periodic; z is periodic (zbc = 0) or bounded by free-slip walls (zbc = 1):
 * u, v, nu mirrored evenly, w mirrored oddly with w = 0 on both wall faces.
 * Non-uniform z uses index-space interpolation weights and divides flux
 * differences by dz_k (u, v) or dzh_k (w).
 *
 * Every loop is naive: each face flux is evaluated afresh for each point that
 * needs it.  Built with -ffp-contract=off so no fused multiply-add is formed.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- layout */

typedef struct {
    int nx, ny, nz, g;
    int zbc;               /* 0 periodic in z, 1 walls */
    double dx, dy;
    const double *dz;      /* nz + 2g, dz_k  = zh_{k+1} - zh_k, index k + g */
    const double *dzh;     /* nz + 2g, dzh_k = z_k - z_{k-1},   index k + g */
} ogrid;

/* padded array index in the oracle's own layout: x fastest, no alignment */
static size_t P(const ogrid *G, int i, int j, int k)
{
    size_t NX = (size_t)G->nx + 2 * G->g, NY = (size_t)G->ny + 2 * G->g;
    return (size_t)(i + G->g) + NX * ((size_t)(j + G->g) + NY * (size_t)(k + G->g));
}

/* ------------------------------------------------------- vertical profile */

/*
 * Vertical spacings from the face heights zh_0..zh_nz.
 * dz_k = zh_{k+1} - zh_k and z_k = (zh_k + zh_{k+1})/2 on the interior;
 * ghost levels: walls mirror the grid about the wall faces, periodic z wraps
 * it by the domain height.  dzh_k = z_k - z_{k-1} for every level.
 */
void or_zprofile(int nz, int g, int zbc, const double *zh, double *dz, double *dzh)
{
    int n = nz + 2 * g;
    double *zc = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *zf = (double *)malloc(sizeof(double) * (size_t)(n + 2));
    double L = zh[nz] - zh[0];
    /* faces zf[k+g] = zh_k for k in [-g, nz+g] */
    for (int k = -g; k <= nz + g; ++k) {
        double v;
        if (k >= 0 && k <= nz) v = zh[k];
        else if (zbc == 1) v = (k < 0) ? 2.0 * zh[0] - zh[-k] : 2.0 * zh[nz] - zh[2 * nz - k];
        else v = (k < 0) ? zh[k + nz] - L : zh[k - nz] + L;
        zf[k + g] = v;
    }
    for (int k = -g; k < nz + g; ++k) {
        dz[k + g] = zf[k + 1 + g] - zf[k + g];
        zc[k + g] = 0.5 * (zf[k + g] + zf[k + 1 + g]);
    }
    for (int k = -g; k < nz + g; ++k) {
        if (k == -g) {
            /* one level further down, from the same mirrored/wrapped faces */
            double zlo;
            int kk = -g - 1;
            double fa, fb;
            if (zbc == 1) { fa = 2.0 * zh[0] - zh[-kk]; fb = 2.0 * zh[0] - zh[-kk - 1]; }
            else { fa = zh[kk + nz] - L; fb = zh[kk + 1 + nz] - L; }
            zlo = 0.5 * (fa + fb);
            dzh[k + g] = zc[k + g] - zlo;
        } else {
            dzh[k + g] = zc[k + g] - zc[k - 1 + g];
        }
    }
    free(zc);
    free(zf);
}

/* ------------------------------------------------------------- ghost fill */

static int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

/*
 * Fill the ghost cells of one padded field from its interior.
 * odd = 0: periodic, or even mirror a(-1-m) = a(m) at the walls (u, v, nu).
 * odd = 1: periodic, or odd mirror at the walls with w(0) = w(nz) = 0 and
 *          w(-m) = -w(m), w(nz+m) = -w(nz-m) (w).
 * Each ghost point maps straight to an interior point (each axis mapped on
 * its own), so the result does not depend on the order of the faces.
 */
void or_fill_ghosts(int nx, int ny, int nz, int g, int zbc, int odd, double *a)
{
    ogrid G = {nx, ny, nz, g, zbc, 0, 0, 0, 0};
    for (int k = -g; k < nz + g; ++k)
        for (int j = -g; j < ny + g; ++j)
            for (int i = -g; i < nx + g; ++i) {
                int inside = i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz;
                if (inside) continue;
                int si = wrap(i, nx), sj = wrap(j, ny), sk = k;
                double sign = 1.0;
                if (zbc == 0) {
                    sk = wrap(k, nz);
                } else if (!odd) {
                    if (k < 0) sk = -1 - k;
                    else if (k >= nz) sk = 2 * nz - 1 - k;
                } else {
                    if (k < 0) { sk = -k; sign = -1.0; }
                    else if (k == nz) { a[P(&G, i, j, k)] = 0.0; continue; }
                    else if (k > nz) { sk = 2 * nz - k; sign = -1.0; }
                }
                a[P(&G, i, j, k)] = sign * a[P(&G, si, sj, sk)];
            }
}

/* ------------------------------------------------------ 1D interpolation */

/* 6-point centred interpolation to the mid point of a[2], a[3] */
static double I6(const double a[6])
{
    return (a[0] - 8.0 * a[1] + 37.0 * a[2] + 37.0 * a[3] - 8.0 * a[4] + a[5]) / 60.0;
}

/* 6-point dissipative correction; I6 + D6 is the upwind-biased 5th-order form */
static double D6(const double a[6])
{
    return (a[0] - 5.0 * a[1] + 10.0 * a[2] - 10.0 * a[3] + 5.0 * a[4] - a[5]) / 60.0;
}

/* face flux of the advected quantity a (6 values around the face) by velocity U */
static double flux(int adv, double U, const double a[6])
{
    if (adv == 2) return U * ((a[2] + a[3]) / 2.0);
    if (adv == 6) return U * I6(a);
    return U * I6(a) + fabs(U) * D6(a);
}

/* -------------------------------------------------------- advection terms */

typedef struct {
    const ogrid *G;
    const double *u, *v, *w;
    int adv;
} actx;

#define U_(i, j, k) (C->u[P(C->G, (i), (j), (k))])
#define V_(i, j, k) (C->v[P(C->G, (i), (j), (k))])
#define W_(i, j, k) (C->w[P(C->G, (i), (j), (k))])

/* six values of field f along axis ax starting at offset s0 from (i,j,k) */
static void window(const actx *C, const double *f, int ax, int i, int j, int k, int s0, double a[6])
{
    for (int q = 0; q < 6; ++q) {
        int o = s0 + q;
        int ii = i + (ax == 0 ? o : 0), jj = j + (ax == 1 ? o : 0), kk = k + (ax == 2 ? o : 0);
        a[q] = f[P(C->G, ii, jj, kk)];
    }
}

/* u-momentum fluxes, u point (i,j,k) at (xh_i, y_j, z_k) */
static double Fux(const actx *C, int i, int j, int k)  /* at centre x_i */
{
    double a[6];
    window(C, C->u, 0, i, j, k, -2, a);             /* u(i-2 .. i+3) */
    return flux(C->adv, (U_(i, j, k) + U_(i + 1, j, k)) / 2.0, a);
}
static double Fuy(const actx *C, int i, int j, int k)  /* at edge (xh_i, yh_j) */
{
    double a[6];
    window(C, C->u, 1, i, j, k, -3, a);             /* u(j-3 .. j+2) */
    return flux(C->adv, (V_(i - 1, j, k) + V_(i, j, k)) / 2.0, a);
}
static double Fuz(const actx *C, int i, int j, int k)  /* at edge (xh_i, zh_k) */
{
    double a[6];
    window(C, C->u, 2, i, j, k, -3, a);             /* u(k-3 .. k+2) */
    return flux(C->adv, (W_(i - 1, j, k) + W_(i, j, k)) / 2.0, a);
}

/* v-momentum fluxes, v point (i,j,k) at (x_i, yh_j, z_k) */
static double Fvx(const actx *C, int i, int j, int k)  /* at edge (xh_i, yh_j) */
{
    double a[6];
    window(C, C->v, 0, i, j, k, -3, a);
    return flux(C->adv, (U_(i, j - 1, k) + U_(i, j, k)) / 2.0, a);
}
static double Fvy(const actx *C, int i, int j, int k)  /* at centre y_j */
{
    double a[6];
    window(C, C->v, 1, i, j, k, -2, a);
    return flux(C->adv, (V_(i, j, k) + V_(i, j + 1, k)) / 2.0, a);
}
static double Fvz(const actx *C, int i, int j, int k)  /* at edge (yh_j, zh_k) */
{
    double a[6];
    window(C, C->v, 2, i, j, k, -3, a);
    return flux(C->adv, (W_(i, j - 1, k) + W_(i, j, k)) / 2.0, a);
}

/* w-momentum fluxes, w point (i,j,k) at (x_i, y_j, zh_k) */
static double Fwx(const actx *C, int i, int j, int k)  /* at edge (xh_i, zh_k) */
{
    double a[6];
    window(C, C->w, 0, i, j, k, -3, a);
    return flux(C->adv, (U_(i, j, k - 1) + U_(i, j, k)) / 2.0, a);
}
static double Fwy(const actx *C, int i, int j, int k)  /* at edge (yh_j, zh_k) */
{
    double a[6];
    window(C, C->w, 1, i, j, k, -3, a);
    return flux(C->adv, (V_(i, j, k - 1) + V_(i, j, k)) / 2.0, a);
}
static double Fwz(const actx *C, int i, int j, int k)  /* at centre z_k */
{
    double a[6];
    window(C, C->w, 2, i, j, k, -2, a);
    return flux(C->adv, (W_(i, j, k) + W_(i, j, k + 1)) / 2.0, a);
}

/* ----------------------------------------------------- diffusion, const nu */

static double lap_uv(const ogrid *G, const double *a, int i, int j, int k)
{
    double c = a[P(G, i, j, k)];
    double dxx = (a[P(G, i + 1, j, k)] - 2.0 * c + a[P(G, i - 1, j, k)]) / (G->dx * G->dx);
    double dyy = (a[P(G, i, j + 1, k)] - 2.0 * c + a[P(G, i, j - 1, k)]) / (G->dy * G->dy);
    double up = (a[P(G, i, j, k + 1)] - c) / G->dzh[k + 1 + G->g];
    double dn = (c - a[P(G, i, j, k - 1)]) / G->dzh[k + G->g];
    return dxx + dyy + (up - dn) / G->dz[k + G->g];
}

static double lap_w(const ogrid *G, const double *a, int i, int j, int k)
{
    double c = a[P(G, i, j, k)];
    double dxx = (a[P(G, i + 1, j, k)] - 2.0 * c + a[P(G, i - 1, j, k)]) / (G->dx * G->dx);
    double dyy = (a[P(G, i, j + 1, k)] - 2.0 * c + a[P(G, i, j - 1, k)]) / (G->dy * G->dy);
    double up = (a[P(G, i, j, k + 1)] - c) / G->dz[k + G->g];
    double dn = (c - a[P(G, i, j, k - 1)]) / G->dz[k - 1 + G->g];
    return dxx + dyy + (up - dn) / G->dzh[k + G->g];
}

/* ------------------------------------------------ diffusion, variable nu */

typedef struct {
    const ogrid *G;
    const double *u, *v, *w, *n;
} dctx;

#define DU(i, j, k) (D->u[P(D->G, (i), (j), (k))])
#define DV(i, j, k) (D->v[P(D->G, (i), (j), (k))])
#define DW(i, j, k) (D->w[P(D->G, (i), (j), (k))])
#define DN(i, j, k) (D->n[P(D->G, (i), (j), (k))])
#define DZI(k) (1.0 / D->G->dz[(k) + D->G->g])
#define DZHI(k) (1.0 / D->G->dzh[(k) + D->G->g])

/* nu on the edges: (xh,yh,z), (xh,y,zh), (x,yh,zh); 4-point averages */
static double nxy(const dctx *D, int i, int j, int k)
{ return (DN(i - 1, j - 1, k) + DN(i, j - 1, k) + DN(i - 1, j, k) + DN(i, j, k)) / 4.0; }
static double nxz(const dctx *D, int i, int j, int k)
{ return (DN(i - 1, j, k - 1) + DN(i, j, k - 1) + DN(i - 1, j, k) + DN(i, j, k)) / 4.0; }
static double nyz(const dctx *D, int i, int j, int k)
{ return (DN(i, j - 1, k - 1) + DN(i, j, k - 1) + DN(i, j - 1, k) + DN(i, j, k)) / 4.0; }

/* stresses; tau_xy = nu (du/dy + dv/dx) on (xh_i, yh_j, z_k), etc. */
static double Sxx(const dctx *D, int i, int j, int k)  /* centre */
{ return 2.0 * DN(i, j, k) * (DU(i + 1, j, k) - DU(i, j, k)) / D->G->dx; }
static double Syy(const dctx *D, int i, int j, int k)
{ return 2.0 * DN(i, j, k) * (DV(i, j + 1, k) - DV(i, j, k)) / D->G->dy; }
static double Szz(const dctx *D, int i, int j, int k)
{ return 2.0 * DN(i, j, k) * (DW(i, j, k + 1) - DW(i, j, k)) / D->G->dz[k + D->G->g]; }
static double Sxy(const dctx *D, int i, int j, int k)
{
    return nxy(D, i, j, k) * ((DU(i, j, k) - DU(i, j - 1, k)) / D->G->dy +
                              (DV(i, j, k) - DV(i - 1, j, k)) / D->G->dx);
}
static double Sxz(const dctx *D, int i, int j, int k)
{
    return nxz(D, i, j, k) * ((DU(i, j, k) - DU(i, j, k - 1)) / D->G->dzh[k + D->G->g] +
                              (DW(i, j, k) - DW(i - 1, j, k)) / D->G->dx);
}
static double Syz(const dctx *D, int i, int j, int k)
{
    return nyz(D, i, j, k) * ((DV(i, j, k) - DV(i, j, k - 1)) / D->G->dzh[k + D->G->g] +
                              (DW(i, j, k) - DW(i, j - 1, k)) / D->G->dy);
}

/* ------------------------------------------------------------ tendencies */

/*
 * ut, vt, wt on interior levels k0 <= k < k1 (arrays of (k1-k0)*ny*nx, x
 * fastest) from padded u, v, w (and nu for diff = 2) whose ghosts are already
 * filled.  With walls, wt = 0 at k = 0.
 */
void or_tendency(int nx, int ny, int nz, int g, int zbc, double dx, double dy,
                 const double *dz, const double *dzh, int adv, int diff, double nu,
                 const double *u, const double *v, const double *w, const double *nuf,
                 int k0, int k1, double *ut, double *vt, double *wt)
{
    ogrid G = {nx, ny, nz, g, zbc, dx, dy, dz, dzh};
    actx A = {&G, u, v, w, adv};
    dctx D = {&G, u, v, w, nuf};
    const actx *C = &A;
    /* Only the timing build (-fopenmp, liboracle_omp) splits the rows among
     * threads; every point is computed by the same code in either build, so
     * the results are identical. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t o = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * (size_t)(k - k0));
                double tu = 0.0, tv = 0.0, tw = 0.0;
                double dzk = dz[k + g], dzhk = dzh[k + g];
                int wall_w = (zbc == 1 && k == 0);
                if (adv) {
                    tu += -(Fux(C, i, j, k) - Fux(C, i - 1, j, k)) / dx
                          - (Fuy(C, i, j + 1, k) - Fuy(C, i, j, k)) / dy
                          - (Fuz(C, i, j, k + 1) - Fuz(C, i, j, k)) / dzk;
                    tv += -(Fvx(C, i + 1, j, k) - Fvx(C, i, j, k)) / dx
                          - (Fvy(C, i, j, k) - Fvy(C, i, j - 1, k)) / dy
                          - (Fvz(C, i, j, k + 1) - Fvz(C, i, j, k)) / dzk;
                    if (!wall_w)
                        tw += -(Fwx(C, i + 1, j, k) - Fwx(C, i, j, k)) / dx
                              - (Fwy(C, i, j + 1, k) - Fwy(C, i, j, k)) / dy
                              - (Fwz(C, i, j, k) - Fwz(C, i, j, k - 1)) / dzhk;
                }
                if (diff == 1) {
                    tu += nu * lap_uv(&G, u, i, j, k);
                    tv += nu * lap_uv(&G, v, i, j, k);
                    if (!wall_w) tw += nu * lap_w(&G, w, i, j, k);
                } else if (diff == 2) {
                    const dctx *Dp = &D;
                    tu += (Sxx(Dp, i, j, k) - Sxx(Dp, i - 1, j, k)) / dx
                          + (Sxy(Dp, i, j + 1, k) - Sxy(Dp, i, j, k)) / dy
                          + (Sxz(Dp, i, j, k + 1) - Sxz(Dp, i, j, k)) / dzk;
                    tv += (Sxy(Dp, i + 1, j, k) - Sxy(Dp, i, j, k)) / dx
                          + (Syy(Dp, i, j, k) - Syy(Dp, i, j - 1, k)) / dy
                          + (Syz(Dp, i, j, k + 1) - Syz(Dp, i, j, k)) / dzk;
                    if (!wall_w)
                        tw += (Sxz(Dp, i + 1, j, k) - Sxz(Dp, i, j, k)) / dx
                              + (Syz(Dp, i, j + 1, k) - Syz(Dp, i, j, k)) / dy
                              + (Szz(Dp, i, j, k) - Szz(Dp, i, j, k - 1)) / dzhk;
                }
                ut[o] = tu;
                vt[o] = tv;
                wt[o] = tw;
            }
}

/* ------------------------------------------------- Smagorinsky viscosity */

/*
 * Eddy viscosity of the Smagorinsky model at cell centres of interior levels
 * k0 <= k < k1 (array of (k1-k0)*ny*nx, x fastest), from padded u, v, w
 * whose ghosts are filled (one ghost cell suffices):
 *
 *   nu = (cs * delta_k)^2 * sqrt(2 S_ij S_ij),  delta_k = (dx dy dz_k)^(1/3),
 *   S_ij = (d_i u_j + d_j u_i) / 2.
 *
 * The paper names the model ("Smagorinsky diffusion", Sec. 5.2) but prints no
 * formula; this is the textbook model discretised on the C grid.  The normal
 * strains live at the cell centre.  Each shear strain lives on cell edges
 * (Sxy on (xh, yh, z), Sxz on (xh, y, zh), Syz on (x, yh, zh)); its square
 * enters as the mean over the four edges of the cell, so that
 *
 *   2 S_ij S_ij = 2 (Sxx^2 + Syy^2 + Szz^2) + 4 (<Sxy^2> + <Sxz^2> + <Syz^2>).
 */
static double exy(const dctx *D, int i, int j, int k)  /* Sxy on (xh_i, yh_j, z_k) */
{
    return 0.5 * ((DU(i, j, k) - DU(i, j - 1, k)) / D->G->dy +
                  (DV(i, j, k) - DV(i - 1, j, k)) / D->G->dx);
}
static double exz(const dctx *D, int i, int j, int k)  /* Sxz on (xh_i, y_j, zh_k) */
{
    return 0.5 * ((DU(i, j, k) - DU(i, j, k - 1)) / D->G->dzh[k + D->G->g] +
                  (DW(i, j, k) - DW(i - 1, j, k)) / D->G->dx);
}
static double eyz(const dctx *D, int i, int j, int k)  /* Syz on (x_i, yh_j, zh_k) */
{
    return 0.5 * ((DV(i, j, k) - DV(i, j, k - 1)) / D->G->dzh[k + D->G->g] +
                  (DW(i, j, k) - DW(i, j - 1, k)) / D->G->dy);
}

void or_smagorinsky(int nx, int ny, int nz, int g, double dx, double dy, const double *dz,
                    const double *dzh, double cs, const double *u, const double *v,
                    const double *w, int k0, int k1, double *nu)
{
    ogrid G = {nx, ny, nz, g, 0, dx, dy, dz, dzh};
    dctx Dc = {&G, u, v, w, NULL};
    const dctx *D = &Dc;
    for (int k = k0; k < k1; ++k) {
        double delta = cbrt(dx * dy * dz[k + g]);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double sxx = (DU(i + 1, j, k) - DU(i, j, k)) / dx;
                double syy = (DV(i, j + 1, k) - DV(i, j, k)) / dy;
                double szz = (DW(i, j, k + 1) - DW(i, j, k)) / dz[k + g];
                double mxy = 0.0, mxz = 0.0, myz = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        double e1 = exy(D, i + a, j + b, k);
                        double e2 = exz(D, i + a, j, k + b);
                        double e3 = eyz(D, i, j + a, k + b);
                        mxy += e1 * e1 / 4.0;
                        mxz += e2 * e2 / 4.0;
                        myz += e3 * e3 / 4.0;
                    }
                double s2 = 2.0 * (sxx * sxx + syy * syy + szz * szz) + 4.0 * (mxy + mxz + myz);
                size_t o = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * (size_t)(k - k0));
                nu[o] = (cs * delta) * (cs * delta) * sqrt(s2);
            }
    }
}

/* ------------------------------------------------------------ diagnostics */

/*
 * FP64 diagnostics of one tendency t against a reference r over n values:
 * out = {max|t-r|, sqrt(mean (t-r)^2), max|r|, sqrt(mean r^2), sum t, sum t*wgt}
 * wgt (length n, may be NULL for all ones) carries dz for mass-weighted sums.
 */
void or_diag(size_t n, const double *t, const double *r, const double *wgt, double out[6])
{
    double emax = 0.0, e2 = 0.0, rmax = 0.0, r2 = 0.0, s = 0.0, sw = 0.0;
    for (size_t q = 0; q < n; ++q) {
        double e = t[q] - (r ? r[q] : 0.0);
        double rv = r ? r[q] : 0.0;
        if (fabs(e) > emax) emax = fabs(e);
        if (fabs(rv) > rmax) rmax = fabs(rv);
        e2 += e * e;
        r2 += rv * rv;
        s += t[q];
        sw += t[q] * (wgt ? wgt[q] : 1.0);
    }
    out[0] = emax;
    out[1] = n ? sqrt(e2 / (double)n) : 0.0;
    out[2] = rmax;
    out[3] = n ? sqrt(r2 / (double)n) : 0.0;
    out[4] = s;
    out[5] = sw;
}

/* Threads of the OpenMP timing build (the serial build has one). */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
