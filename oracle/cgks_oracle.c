/*
 * FP64 CPU oracle of the ASE-DFF compact gas-kinetic scheme: the per-stage
 * face evaluation (reconstruction, DFF, kinetic flux and interface state).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference leg of bench.py may load it.  It shares no code,
 * header or table generator with the CUDA library.
 *
 * Written as plain loops in the paper's order:
 *   Sec. 3.3 Step 1   tangential ASE-DFF -> line averages at Gauss lines
 *   Sec. 3.3 Step 2   normal ASE-DFF (Algorithm 1, Eq. 3.3-3.19)
 *   Sec. 3.3 Step 3   tangential derivatives at face Gauss points
 *   Eq. 3.1-3.2       discontinuity strength sigma at every face Gauss point
 *   Eq. 2.7-2.8       kinetic weighting and micro-slopes (Step 4)
 *   Eq. 2.6, 2.11, 2.12, 2.15  time-integrated flux and interface state
 * The time stepping (Eq. 2.13-2.30) is done by the Python side of the oracle.
 *
 * Compile: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_FIXED = 2, BC_REFLECTIVE = 3, BC_NOSLIP = 4,
       BC_INFLOW = 5, BC_INFLOW_REFLECTIVE = 6 };
enum { K_W = 0, K_WX = 1, K_WY = 2, K_WXL = 3, K_WYL = 4 };
enum { ST_S0 = 0, ST_S1 = 1, ST_S2 = 2, ST_R5 = 3, ST_R7 = 4, ST_R9 = 5 };
/* flag bits */
enum { FL_NONPHYS = 1 };

#define NMOM 12

typedef struct {
    int dim, order, m, nx, ny;
    int bc[4];       /* xlo, xhi, ylo, yhi */
    int tau_mode;    /* 0: tau = 0, 1: tau = c1 dt + c2 |pl-pr|/(pl+pr) dt, 2: mu/p0 + c2 |pl-pr|/(pl+pr) dt */
    int step3;       /* 0: Lagrange through 3m face points, 1: 3-point central */
    int flux_tt;     /* 1: keep the t^2/2 a_tt g0 term of Eq. 2.6 in the flux integral */
    int dff_faces;   /* 0: all faces of the stencil's cells, 1: interior faces only */
    int step3_deg;   /* Step 3 fit degree through the 3m points (0: 3m-1, interpolation) */
    double dx, dy, gamma;
    double sigma_thres, gamma_hi, gamma_lo, weno_eps, c1, c2;
    double mu;       /* dynamic viscosity (tau_mode 2) */
    double x0, y0;   /* lower-left corner of the mesh */
    double tb;       /* time at which prescribed ghost states are taken (this stage's) */
    /* prescribed ghost states (conservative) per side: [0] where the
     * coordinate along the side is below split(t) = bcx[0] + bcx[1] t, [1] beyond */
    double bcs[4][2][4];
    double bcx[4][2];
    int pt_fallback; /* 1: first-order fallback at non-physical face points (a flagged option) */
} OParams;

typedef struct {
    const OParams *P;
    const double *T;   /* [6][9][10] stencil polynomial tables */
    const double *gx;  /* Gauss nodes on [-1/2, 1/2] */
    const double *W, *Wx, *Wy, *Wxl, *Wyl, *sx, *sy;
    const double *ghost; /* 1-D fixed BC: [2 sides][3 layers][2 fields][3 vars] */
    int nv;
    double K;          /* internal degrees of freedom */
} Ctx;

static int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* ------------------------------------------------------------------ */
/* Boundary handling: ghost cells and ghost faces                      */
/* ------------------------------------------------------------------ */

/* Cell field value with the ghost-cell rule applied direction by direction
 * (x first): periodic wraps; transmissive copies the nearest interior cell and
 * zeroes the slopes normal to that boundary; fixed (1-D) reads the stored
 * ghost; a wall mirrors; inflow holds a prescribed state with zero slopes. */
static int is_wall(int bc) { return bc == BC_REFLECTIVE || bc == BC_NOSLIP; }

/* Sign of a mirrored ghost value across a wall whose normal is the x axis
 * (normal = 0) or the y axis (normal = 1).  Reflection x -> -x maps a field
 * q to S q(-x), with S reversing the normal momentum (slip wall) or both
 * momenta (no-slip wall); a derivative along the normal picks up one more
 * sign, a derivative along the wall none. */
static double wall_sign(int kind, int v, int normal, int bc, int nv)
{
    int rev = (v == 1 + normal) || (bc == BC_NOSLIP && v >= 1 && v <= nv - 2);
    int dnormal = normal == 0 ? (kind == K_WX || kind == K_WXL) : (kind == K_WY || kind == K_WYL);
    return (rev ^ dnormal) ? -1.0 : 1.0;
}

/* Prescribed ghost states (inflow sides): is the centre of ghost row or
 * column k, taken along side `side`, below that side's split point at the
 * stage time, split(t) = bcx[0] + bcx[1] t?  Below it the ghost cell holds
 * bcs[side][0], beyond it bcs[side][1] (or, on a side that is a slip wall in
 * part, the mirror image). */
static int below_split(const OParams *P, int side, int k)
{
    double s = side < 2 ? P->y0 + (k + 0.5) * P->dy : P->x0 + (k + 0.5) * P->dx;
    return s < P->bcx[side][0] + P->bcx[side][1] * P->tb;
}

static double cellval(const Ctx *c, int kind, int v, int l, int i, int j)
{
    const OParams *P = c->P;
    int nx = P->nx, ny = P->ny, zero = 0;
    double sgn = 1.0;
    if (i < 0 || i >= nx) {
        int side = i < 0 ? 0 : 1;
        int bc = P->bc[side];
        if (bc == BC_PERIODIC) {
            i = imod(i, nx);
        } else if (bc == BC_FIXED) {
            int layer = side == 0 ? (-1 - i) : (i - nx);
            int f = kind == K_W ? 0 : 1;
            return c->ghost[((side * 3 + layer) * 2 + f) * 3 + v];
        } else if (bc == BC_INFLOW || (bc == BC_INFLOW_REFLECTIVE && below_split(P, side, j))) {
            /* prescribed state by the row's centre, zero slopes */
            return kind == K_W ? P->bcs[side][below_split(P, side, j) ? 0 : 1][v] : 0.0;
        } else if (is_wall(bc) || bc == BC_INFLOW_REFLECTIVE) {
            /* ghost cell -1-k mirrors cell k; lines across x (Wy_line) swap ends */
            i = i < 0 ? -1 - i : 2 * nx - 1 - i;
            sgn *= wall_sign(kind, v, 0, bc, c->nv);
            if (kind == K_WYL) l = P->m - 1 - l;
        } else {
            i = i < 0 ? 0 : nx - 1;
            if (kind == K_WX || kind == K_WXL) zero = 1;
        }
    }
    if (j < 0 || j >= ny) {
        int side = j < 0 ? 2 : 3;
        int bc = P->bc[side];
        if (bc == BC_INFLOW || (bc == BC_INFLOW_REFLECTIVE && below_split(P, side, i)))
            /* prescribed state by the column's centre (after the x rule), zero slopes */
            return kind == K_W ? sgn * P->bcs[side][below_split(P, side, i) ? 0 : 1][v] : 0.0;
        if (bc == BC_PERIODIC) {
            j = imod(j, ny);
        } else if (is_wall(bc) || bc == BC_INFLOW_REFLECTIVE) {
            j = j < 0 ? -1 - j : 2 * ny - 1 - j;
            sgn *= wall_sign(kind, v, 1, bc, c->nv);
            if (kind == K_WXL) l = P->m - 1 - l;
        } else {
            j = j < 0 ? 0 : ny - 1;
            if (kind == K_WY || kind == K_WYL) zero = 1;
        }
    }
    if (zero) return 0.0;
    size_t plane = (size_t)nx * ny;
    size_t idx = (size_t)j * nx + i;
    double val;
    switch (kind) {
    case K_W: val = c->W[v * plane + idx]; break;
    case K_WX: val = c->Wx[v * plane + idx]; break;
    case K_WY: val = c->Wy[v * plane + idx]; break;
    case K_WXL: val = c->Wxl[((size_t)l * c->nv + v) * plane + idx]; break;
    default: val = c->Wyl[((size_t)l * c->nv + v) * plane + idx]; break;
    }
    return sgn * val;
}
/* Face sigma beyond a wall (or a side that is a wall in part) mirrors the
 * interior face (face 0 is the wall); beyond other sides it is 0 at the faces
 * normal to the side and copies the nearest row or column along it. */
static double sigx(const Ctx *c, int f, int j)
{
    const OParams *P = c->P;
    int nx = P->nx, ny = P->ny;
    if (f < 0 || f > nx) {
        int bc = P->bc[f < 0 ? 0 : 1];
        if (bc == BC_PERIODIC) f = imod(f, nx);
        else if (is_wall(bc) || bc == BC_INFLOW_REFLECTIVE) f = f < 0 ? -f : 2 * nx - f;
        else return 0.0;
    }
    if (j < 0 || j >= ny) {
        int bc = P->bc[j < 0 ? 2 : 3];
        if (bc == BC_PERIODIC) j = imod(j, ny);
        else if (is_wall(bc) || bc == BC_INFLOW_REFLECTIVE) j = j < 0 ? -1 - j : 2 * ny - 1 - j;
        else j = j < 0 ? 0 : ny - 1;
    }
    return c->sx[(size_t)j * (nx + 1) + f];
}
static double sigy(const Ctx *c, int i, int g)
{
    const OParams *P = c->P;
    int nx = P->nx, ny = P->ny;
    if (g < 0 || g > ny) {
        int bc = P->bc[g < 0 ? 2 : 3];
        if (bc == BC_PERIODIC) g = imod(g, ny);
        else if (is_wall(bc) || bc == BC_INFLOW_REFLECTIVE) g = g < 0 ? -g : 2 * ny - g;
        else return 0.0;
    }
    if (i < 0 || i >= nx) {
        int bc = P->bc[i < 0 ? 0 : 1];
        if (bc == BC_PERIODIC) i = imod(i, nx);
        else if (is_wall(bc) || bc == BC_INFLOW_REFLECTIVE) i = i < 0 ? -1 - i : 2 * nx - 1 - i;
        else i = i < 0 ? 0 : nx - 1;
    }
    return c->sy[(size_t)g * nx + i];
}

/* ------------------------------------------------------------------ */
/* ASE-DFF reconstruction of one cell (Algorithm 1, Eq. 3.3-3.19)      */
/* ------------------------------------------------------------------ */

static double dff_alpha(double A, double thres)
{
    /* Eq. 3.3: alpha = 1 if A < sigma_thres, else sigma_thres / A */
    return A < thres ? 1.0 : thres / A;
}

static void stencil_poly(const Ctx *c, int st, const double d[10], double p[9])
{
    const double *T = c->T + (size_t)st * 90;
    for (int n = 0; n < 9; n++) {
        double s = 0.0;
        for (int k = 0; k < 10; k++) s += T[n * 10 + k] * d[k];
        p[n] = s;
    }
}

/* DFF-scaled polynomial, Eq. 3.5 / 3.19: P = Qbar_i + alpha (p - Qbar_i) */
static void dff_scale(double p[9], double qi, double alpha)
{
    p[0] = qi + alpha * (p[0] - qi);
    for (int n = 1; n < 9; n++) p[n] *= alpha;
}

/* Smoothness indicator, Eq. 3.13, in the unit coordinate:
 * beta = sum_{q=1}^{deg} int_{-1/2}^{1/2} (d^q p / dxi^q)^2 dxi */
static double smoothness(const double p[9], int deg)
{
    double beta = 0.0;
    for (int q = 1; q <= deg; q++) {
        double dq[9] = {0};
        for (int n = q; n <= deg; n++) {
            double f = 1.0;
            for (int r = 0; r < q; r++) f *= (double)(n - r);
            dq[n - q] = f * p[n];
        }
        /* integral of the square over [-1/2, 1/2] */
        for (int a = 0; a <= deg - q; a++)
            for (int b = 0; b <= deg - q; b++) {
                int e = a + b;
                if (e % 2) continue;
                beta += dq[a] * dq[b] * 2.0 * pow(0.5, e + 1) / (e + 1);
            }
    }
    return beta;
}

/* Stencil DFF sums, Eq. 3.3-3.4.  sig[0..5] = sigma of faces i-5/2 ... i+5/2.
 * A stencil's sum runs over every face of every cell it draws data from
 * (dff_faces = 0): S0 {i-1,i} -> i-3/2..i+1/2, S1 {i,i+1} -> i-1/2..i+3/2,
 * r5 = S2 {i-1..i+1} -> i-3/2..i+3/2 (the four terms Eq. 3.3 prints),
 * r7, r9 {i-2..i+2} -> i-5/2..i+5/2; eta = 2 for r9 only (Eq. 3.4).
 * dff_faces = 1 takes only the faces interior to the stencil's span. */
static void stencil_sums(const OParams *P, const double sig[6], double A[6])
{
    if (P->dff_faces == 0) {
        A[ST_S0] = sig[1] + sig[2] + sig[3];
        A[ST_S1] = sig[2] + sig[3] + sig[4];
        A[ST_S2] = sig[1] + sig[2] + sig[3] + sig[4];
        A[ST_R7] = sig[0] + sig[1] + sig[2] + sig[3] + sig[4] + sig[5];
    } else {
        A[ST_S0] = sig[2];
        A[ST_S1] = sig[3];
        A[ST_S2] = sig[2] + sig[3];
        A[ST_R7] = sig[1] + sig[2] + sig[3] + sig[4];
    }
    A[ST_R5] = A[ST_S2];
    A[ST_R9] = 2.0 * A[ST_R7];
}

/* Build the reconstruction polynomial of a cell.
 * d:   [Qbar_{i-2..i+2}, h*Qx_{i-2..i+2}]
 * sig: sigma of faces i-5/2 ... i+5/2 (previous time level)
 * Returns the branch taken: 0 HWENO-AO(5,3), 5/7/9 linear r5/r7/r9. */
static int ase_dff_poly(const Ctx *c, const double d[10], const double sig[6], double P[9])
{
    const OParams *Pp = c->P;
    double thr = Pp->sigma_thres;
    double qi = d[2];
    double A[6];
    stencil_sums(Pp, sig, A);
    double a_r5 = dff_alpha(A[ST_R5], thr);
    double a_s0 = dff_alpha(A[ST_S0], thr);
    double a_s1 = dff_alpha(A[ST_S1], thr);
    double a_s2 = dff_alpha(A[ST_S2], thr);
    double a_r7 = dff_alpha(A[ST_R7], thr);
    double a_r9 = dff_alpha(A[ST_R9], thr);

    int branch, st = ST_R5;
    double alpha = 1.0;
    if (a_r5 < 1.0) {
        branch = 0;
    } else if (Pp->order == 5) {
        branch = 5; st = ST_R5; alpha = a_r5;
    } else if (a_r7 < 1.0) {
        branch = 5; st = ST_R5; alpha = a_r5;
    } else if (Pp->order == 7) {
        branch = 7; st = ST_R7; alpha = a_r7;
    } else if (a_r9 < 1.0) {
        branch = 7; st = ST_R7; alpha = a_r7;
    } else {
        branch = 9; st = ST_R9; alpha = a_r9;
    }
    if (branch != 0) {
        stencil_poly(c, st, d, P);
        dff_scale(P, qi, alpha);
        return branch;
    }
    /* HWENO-AO(5,3) with DFF-scaled sub-polynomials, Eq. 3.11-3.17, 3.19 */
    double pk[4][9];
    const int sts[4] = {ST_S0, ST_S1, ST_S2, ST_R5};
    const double al[4] = {a_s0, a_s1, a_s2, a_r5};
    const int deg[4] = {2, 2, 2, 4};
    double gh = Pp->gamma_hi, gl = Pp->gamma_lo;
    /* linear weights: big stencil gamma_Hi; central 3-cell stencil
     * (1-gamma_Hi) gamma_Lo; the two 2-cell stencils share the rest */
    double g[4];
    g[3] = gh;
    g[2] = (1.0 - gh) * gl;
    g[0] = (1.0 - gh) * (1.0 - gl) * 0.5;
    g[1] = g[0];
    double beta[4];
    for (int k = 0; k < 4; k++) {
        stencil_poly(c, sts[k], d, pk[k]);
        dff_scale(pk[k], qi, al[k]);
        beta[k] = smoothness(pk[k], deg[k]);
    }
    double tz = (fabs(beta[3] - beta[0]) + fabs(beta[3] - beta[1]) + fabs(beta[3] - beta[2])) / 3.0;
    double w[4], ws = 0.0;
    for (int k = 0; k < 4; k++) {
        double q = tz / (beta[k] + Pp->weno_eps);
        w[k] = g[k] * (1.0 + q * q);
        ws += w[k];
    }
    for (int k = 0; k < 4; k++) w[k] /= ws;
    for (int n = 0; n < 9; n++) {
        double hi = pk[3][n] / g[3];
        for (int k = 0; k < 3; k++) hi -= g[k] / g[3] * pk[k][n];
        double v = w[3] * hi;
        for (int k = 0; k < 3; k++) v += w[k] * pk[k][n];
        P[n] = v;
    }
    return 0;
}

static double poly_der(const double P[9], double xi, int nd)
{
    double s = 0.0;
    for (int n = nd; n < 9; n++) {
        double f = 1.0;
        for (int r = 0; r < nd; r++) f *= (double)(n - r);
        s += f * P[n] * pow(xi, n - nd);
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Maxwellian moments (per unit density)                               */
/* ------------------------------------------------------------------ */

typedef struct {
    double rho, U, V, lam;
    double mu[3][NMOM]; /* <u^n>: 0 full range, 1 u>0, 2 u<0 */
    double mv[NMOM];    /* <v^n> full range */
    double mxi[4];      /* <(xi^2)^c> */
} Maxw;

static int maxw_from_W(const Ctx *c, const double *W, Maxw *M)
{
    int dim = c->P->dim;
    double rho = W[0];
    double U = W[1] / rho;
    double V = dim == 2 ? W[2] / rho : 0.0;
    double E = W[dim + 1];
    double p = (c->P->gamma - 1.0) * (E - 0.5 * rho * (U * U + V * V));
    M->rho = rho; M->U = U; M->V = V;
    M->lam = rho / (2.0 * p);
    int ok = rho > 0.0 && p > 0.0 && isfinite(rho) && isfinite(p);
    double lam = M->lam;
    /* full range: <u^0> = 1, <u^1> = U, <u^{n+2}> = U<u^{n+1}> + (n+1)/(2 lam) <u^n> */
    double sl = sqrt(lam);
    double e = exp(-lam * U * U) / (2.0 * sqrt(M_PI * lam));
    M->mu[0][0] = 1.0; M->mu[0][1] = U;
    M->mu[1][0] = 0.5 * erfc(-sl * U); M->mu[1][1] = U * M->mu[1][0] + e;
    M->mu[2][0] = 0.5 * erfc(sl * U);  M->mu[2][1] = U * M->mu[2][0] - e;
    for (int r = 0; r < 3; r++)
        for (int n = 0; n + 2 < NMOM; n++)
            M->mu[r][n + 2] = U * M->mu[r][n + 1] + (n + 1) / (2.0 * lam) * M->mu[r][n];
    M->mv[0] = 1.0; M->mv[1] = V;
    for (int n = 0; n + 2 < NMOM; n++) M->mv[n + 2] = V * M->mv[n + 1] + (n + 1) / (2.0 * lam) * M->mv[n];
    /* K independent internal components of variance 1/(2 lam) each */
    M->mxi[0] = 1.0;
    for (int q = 1; q < 4; q++) M->mxi[q] = M->mxi[q - 1] * (c->K / 2.0 + (q - 1)) / lam;
    return ok;
}

/* Basis of the collision invariants psi as monomials u^a v^b (xi^2)^s:
 * 1-D: (1, u, (u^2+xi^2)/2);  2-D: (1, u, v, (u^2+v^2+xi^2)/2). */
typedef struct { int n; double c[3]; int a[3], b[3], s[3]; } Poly;

static Poly basis(int dim, int k)
{
    Poly p;
    memset(&p, 0, sizeof p);
    if (k == 0) { p.n = 1; p.c[0] = 1; }
    else if (k == 1) { p.n = 1; p.c[0] = 1; p.a[0] = 1; }
    else if (dim == 2 && k == 2) { p.n = 1; p.c[0] = 1; p.b[0] = 1; }
    else {
        p.c[0] = 0.5; p.a[0] = 2;
        if (dim == 2) { p.n = 3; p.c[1] = 0.5; p.b[1] = 2; p.c[2] = 0.5; p.s[2] = 1; }
        else { p.n = 2; p.c[1] = 0.5; p.s[1] = 1; }
    }
    return p;
}

/* out_i = rho * < (sum_k a_k psi_k) u^pu v^pv psi_i >_range  (a == NULL: the factor is 1) */
static void mom_vec(const Ctx *c, const Maxw *M, int range, const double *a, int pu, int pv, double *out)
{
    int dim = c->P->dim, nv = c->nv;
    for (int i = 0; i < nv; i++) {
        Poly pi = basis(dim, i);
        double s = 0.0;
        for (int k = 0; k < (a ? nv : 1); k++) {
            double ak = a ? a[k] : 1.0;
            if (ak == 0.0) continue;
            Poly pk = a ? basis(dim, k) : basis(dim, 0);
            for (int x = 0; x < pi.n; x++)
                for (int y = 0; y < pk.n; y++) {
                    int eu = pi.a[x] + pk.a[y] + pu;
                    int ev = pi.b[x] + pk.b[y] + pv;
                    int es = pi.s[x] + pk.s[y];
                    s += ak * pi.c[x] * pk.c[y] * M->mu[range][eu] * M->mv[ev] * M->mxi[es];
                }
        }
        out[i] = M->rho * s;
    }
}

/* Solve <a> = b, i.e. the Gram system sum_k rho<psi_k psi_i> a_k = b_i (Eq. 2.8),
 * by Gaussian elimination with partial pivoting. */
static void micro_slope(const Ctx *c, const Maxw *M, const double *b, double *a)
{
    int n = c->nv;
    double A[4][5];
    for (int k = 0; k < n; k++) {
        double e[4] = {0, 0, 0, 0}, col[4];
        e[k] = 1.0;
        mom_vec(c, M, 0, e, 0, 0, col);
        for (int i = 0; i < n; i++) A[i][k] = col[i];
    }
    for (int i = 0; i < n; i++) A[i][n] = b[i];
    for (int col = 0; col < n; col++) {
        int p = col;
        for (int r = col + 1; r < n; r++) if (fabs(A[r][col]) > fabs(A[p][col])) p = r;
        if (p != col) for (int q = 0; q <= n; q++) { double t = A[col][q]; A[col][q] = A[p][q]; A[p][q] = t; }
        for (int r = col + 1; r < n; r++) {
            double f = A[r][col] / A[col][col];
            for (int q = col; q <= n; q++) A[r][q] -= f * A[col][q];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = A[r][n];
        for (int q = r + 1; q < n; q++) s -= A[r][q] * a[q];
        a[r] = s / A[r][r];
    }
}

/* ------------------------------------------------------------------ */
/* Gas-kinetic flux at one face Gauss point, local frame (n, t)        */
/* ------------------------------------------------------------------ */

/* Side data: D[0]=W, D[1]=W_n, D[2]=W_nn, D[3]=W_t, D[4]=W_tt, D[5]=W_nt */
typedef struct { double D[6][4]; } Side;

static void pressure_mach(const Ctx *c, const double *W, double *p, double *man, double *mat)
{
    int dim = c->P->dim;
    double rho = W[0], U = W[1] / rho, V = dim == 2 ? W[2] / rho : 0.0;
    *p = (c->P->gamma - 1.0) * (W[dim + 1] - 0.5 * rho * (U * U + V * V));
    double a = sqrt(c->P->gamma * *p / rho);
    *man = U / a;
    *mat = V / a;
}

/* Eq. 3.2 */
static double sigma_point(const Ctx *c, const double *Wl, const double *Wr)
{
    double pl, pr, mnl, mnr, mtl, mtr;
    pressure_mach(c, Wl, &pl, &mnl, &mtl);
    pressure_mach(c, Wr, &pr, &mnr, &mtr);
    double dp = fabs(pl - pr);
    return dp / pl + dp / pr + (mnl - mnr) * (mnl - mnr) + (mtl - mtr) * (mtl - mtr);
}

/* out[5][nv]: Fbb(dt), Fbb(dt/2), W(0), W(dt/2), W(dt).  Returns 0 if some
 * state on the way had non-positive density or pressure. */
static int kinetic_point(const Ctx *c, const Side *L, const Side *R, double dt, double out[5][4])
{
    const OParams *P = c->P;
    int nv = c->nv, dim = P->dim;
    int nd = dim == 2 ? 5 : 2; /* derivatives carried: n, nn (, t, tt, nt) */
    Maxw Ml, Mr, M0;
    int ok = maxw_from_W(c, L->D[0], &Ml);
    ok &= maxw_from_W(c, R->D[0], &Mr);

    /* micro-slopes of the initial states, <a^k> = dW^k (Eq. 2.8) */
    double al[5][4], ar[5][4];
    const int didx[5] = {1, 2, 3, 4, 5};
    for (int q = 0; q < nd; q++) {
        micro_slope(c, &Ml, L->D[didx[q]], al[q]);
        micro_slope(c, &Mr, R->D[didx[q]], ar[q]);
    }
    /* kinetic weighting, Eq. 2.7 */
    double Q0[4], dQ0[5][4], tl[4], tr[4];
    mom_vec(c, &Ml, 1, NULL, 0, 0, tl);
    mom_vec(c, &Mr, 2, NULL, 0, 0, tr);
    for (int i = 0; i < nv; i++) Q0[i] = tl[i] + tr[i];
    for (int q = 0; q < nd; q++) {
        mom_vec(c, &Ml, 1, al[q], 0, 0, tl);
        mom_vec(c, &Mr, 2, ar[q], 0, 0, tr);
        for (int i = 0; i < nv; i++) dQ0[q][i] = tl[i] + tr[i];
    }
    ok &= maxw_from_W(c, Q0, &M0);

    /* equilibrium micro-slopes and their time derivatives, Eq. 2.8 */
    double ab[5][4];
    for (int q = 0; q < nd; q++) micro_slope(c, &M0, dQ0[q], ab[q]);
    /* ab[0]=a1 (n), ab[1]=a11 (nn), ab[2]=a2 (t), ab[3]=a22 (tt), ab[4]=a12 (nt) */
    double A[4], A1t[4], A2t[4] = {0, 0, 0, 0}, Att[4], rhs[4], t1[4], t2[4];
    mom_vec(c, &M0, 0, ab[0], 1, 0, t1);
    if (dim == 2) mom_vec(c, &M0, 0, ab[2], 0, 1, t2); else memset(t2, 0, sizeof t2);
    for (int i = 0; i < nv; i++) rhs[i] = -(t1[i] + t2[i]);
    micro_slope(c, &M0, rhs, A);
    mom_vec(c, &M0, 0, ab[1], 1, 0, t1);
    if (dim == 2) mom_vec(c, &M0, 0, ab[4], 0, 1, t2); else memset(t2, 0, sizeof t2);
    for (int i = 0; i < nv; i++) rhs[i] = -(t1[i] + t2[i]);
    micro_slope(c, &M0, rhs, A1t);
    if (dim == 2) {
        mom_vec(c, &M0, 0, ab[4], 1, 0, t1);
        mom_vec(c, &M0, 0, ab[3], 0, 1, t2);
        for (int i = 0; i < nv; i++) rhs[i] = -(t1[i] + t2[i]);
        micro_slope(c, &M0, rhs, A2t);
    }
    mom_vec(c, &M0, 0, A1t, 1, 0, t1);
    if (dim == 2) mom_vec(c, &M0, 0, A2t, 0, 1, t2); else memset(t2, 0, sizeof t2);
    for (int i = 0; i < nv; i++) rhs[i] = -(t1[i] + t2[i]);
    micro_slope(c, &M0, rhs, Att);

    /* collision time */
    double tau = 0.0;
    if (P->tau_mode == 1 || P->tau_mode == 2) {
        double pl, pr, p0, dum1, dum2;
        pressure_mach(c, L->D[0], &pl, &dum1, &dum2);
        pressure_mach(c, R->D[0], &pr, &dum1, &dum2);
        /* inviscid: c1 dt; viscous (Sec. 4): mu / p at the face point, p of
           the equilibrium state W0 there */
        pressure_mach(c, Q0, &p0, &dum1, &dum2);
        double base = P->tau_mode == 1 ? P->c1 * dt : P->mu / p0;
        tau = base + P->c2 * fabs(pl - pr) / (pl + pr) * dt;
    }

    /* Eq. 2.6 term by term: (moment source, range, micro-slope factor) */
    /* For the flux every term carries an extra factor u (Eq. 2.12). */
    for (int flux = 0; flux < 2; flux++) {
        int pu = flux;
        double T[11][4];
        double z[4];
        /* 1: g0 */
        mom_vec(c, &M0, 0, NULL, pu, 0, T[0]);
        /* 2: A g0 */
        mom_vec(c, &M0, 0, A, pu, 0, T[1]);
        /* 3: Att g0 */
        mom_vec(c, &M0, 0, Att, pu, 0, T[2]);
        /* 4: (a1 u + a2 v + A) g0 */
        mom_vec(c, &M0, 0, ab[0], pu + 1, 0, T[3]);
        if (dim == 2) { mom_vec(c, &M0, 0, ab[2], pu, 1, z); for (int i = 0; i < nv; i++) T[3][i] += z[i]; }
        for (int i = 0; i < nv; i++) T[3][i] += T[1][i];
        /* 5: (a1t u + a2t v + Att) g0 */
        mom_vec(c, &M0, 0, A1t, pu + 1, 0, T[4]);
        if (dim == 2) { mom_vec(c, &M0, 0, A2t, pu, 1, z); for (int i = 0; i < nv; i++) T[4][i] += z[i]; }
        for (int i = 0; i < nv; i++) T[4][i] += T[2][i];
        /* 6: g0 (times -e^{-t/tau}) */
        memcpy(T[5], T[0], sizeof T[0]);
        /* 7: (a1 u + a2 v) g0 (times t e^{-t/tau}) */
        for (int i = 0; i < nv; i++) T[6][i] = T[3][i] - T[1][i];
        /* 8, 9: g^l H(u), (a1^l u + a2^l v) g^l H(u) */
        mom_vec(c, &Ml, 1, NULL, pu, 0, T[7]);
        mom_vec(c, &Ml, 1, al[0], pu + 1, 0, T[8]);
        if (dim == 2) { mom_vec(c, &Ml, 1, al[2], pu, 1, z); for (int i = 0; i < nv; i++) T[8][i] += z[i]; }
        /* 10, 11: g^r (1-H(u)), (a1^r u + a2^r v) g^r (1-H(u)) */
        mom_vec(c, &Mr, 2, NULL, pu, 0, T[9]);
        mom_vec(c, &Mr, 2, ar[0], pu + 1, 0, T[10]);
        if (dim == 2) { mom_vec(c, &Mr, 2, ar[2], pu, 1, z); for (int i = 0; i < nv; i++) T[10][i] += z[i]; }

        if (flux) {
            /* time integrals over [0, delta] of the coefficients of Eq. 2.6 (Eq. 2.15) */
            for (int h = 0; h < 2; h++) {
                double d = h == 0 ? dt : 0.5 * dt;
                double E0 = 0.0, E1 = 0.0;
                if (tau > 0.0) {
                    double ex = exp(-d / tau);
                    E0 = tau * (1.0 - ex);
                    E1 = tau * tau * (1.0 - ex) - tau * d * ex;
                }
                double C[11] = {d, d * d / 2, P->flux_tt ? d * d * d / 6 : 0.0, -tau * d, -tau * d * d / 2,
                                -E0, E1, E0, -E1, E0, -E1};
                for (int i = 0; i < nv; i++) {
                    double s = 0.0;
                    for (int k = 0; k < 11; k++) s += C[k] * T[k][i];
                    out[h][i] = s;
                }
            }
        } else {
            /* interface state W(t) = int psi f(t) (Eq. 2.11) at t = 0, dt/2, dt */
            for (int h = 0; h < 3; h++) {
                double t = 0.5 * h * dt;
                double e = tau > 0.0 ? exp(-t / tau) : (t == 0.0 ? 1.0 : 0.0);
                double C[11] = {1.0, t, t * t / 2, -tau, -tau * t, -e, t * e, e, -t * e, e, -t * e};
                for (int i = 0; i < nv; i++) {
                    double s = 0.0;
                    for (int k = 0; k < 11; k++) s += C[k] * T[k][i];
                    out[2 + h][i] = s;
                }
            }
        }
    }
    return ok;
}

/* ------------------------------------------------------------------ */
/* Derivative weights for Step 3                                       */
/* ------------------------------------------------------------------ */

/* Least-squares polynomial of degree deg through n points (deg = n-1:
 * interpolation); weights of its first and second derivative at x. */
static void lsq_der(const double *nodes, int n, int deg, double x, double *d1, double *d2)
{
    int q = deg + 1;
    double N[12][12 + 12];
    /* normal matrix V^T V and right-hand sides V^T (identity columns) */
    for (int a = 0; a < q; a++) {
        for (int b = 0; b < q; b++) {
            double s = 0.0;
            for (int k = 0; k < n; k++) s += pow(nodes[k], a) * pow(nodes[k], b);
            N[a][b] = s;
        }
        for (int k = 0; k < n; k++) N[a][q + k] = pow(nodes[k], a);
    }
    for (int col = 0; col < q; col++) {
        int p = col;
        for (int r = col + 1; r < q; r++) if (fabs(N[r][col]) > fabs(N[p][col])) p = r;
        for (int t = 0; t < q + n; t++) { double tmp = N[col][t]; N[col][t] = N[p][t]; N[p][t] = tmp; }
        for (int r = 0; r < q; r++) {
            if (r == col) continue;
            double f = N[r][col] / N[col][col];
            for (int t = 0; t < q + n; t++) N[r][t] -= f * N[col][t];
        }
    }
    for (int k = 0; k < n; k++) {
        double s1 = 0.0, s2 = 0.0;
        for (int a = 0; a < q; a++) {
            double c = N[a][q + k] / N[a][a];
            if (a >= 1) s1 += c * a * pow(x, a - 1);
            if (a >= 2) s2 += c * a * (a - 1) * pow(x, a - 2);
        }
        d1[k] = s1;
        d2[k] = s2;
    }
}

static void lagrange_der(const double *nodes, int n, double x, double *d1, double *d2)
{
    for (int k = 0; k < n; k++) {
        double s1 = 0.0, s2 = 0.0;
        for (int p = 0; p < n; p++) {
            if (p == k) continue;
            double prod = 1.0 / (nodes[k] - nodes[p]);
            for (int q = 0; q < n; q++) {
                if (q == k || q == p) continue;
                prod *= (x - nodes[q]) / (nodes[k] - nodes[q]);
            }
            s1 += prod;
            for (int r = 0; r < n; r++) {
                if (r == k || r == p) continue;
                double pr = 1.0 / ((nodes[k] - nodes[p]) * (nodes[k] - nodes[r]));
                for (int q = 0; q < n; q++) {
                    if (q == k || q == p || q == r) continue;
                    pr *= (x - nodes[q]) / (nodes[k] - nodes[q]);
                }
                s2 += pr;
            }
        }
        d1[k] = s1;
        d2[k] = s2;
    }
}

/* ------------------------------------------------------------------ */
/* Entry points                                                        */
/* ------------------------------------------------------------------ */

static void ctx_init(Ctx *c, const OParams *P, const double *T, const double *gx,
                     const double *W, const double *Wx, const double *Wy, const double *Wxl,
                     const double *Wyl, const double *sx, const double *sy, const double *ghost)
{
    c->P = P; c->T = T; c->gx = gx;
    c->W = W; c->Wx = Wx; c->Wy = Wy; c->Wxl = Wxl; c->Wyl = Wyl;
    c->sx = sx; c->sy = sy; c->ghost = ghost;
    c->nv = P->dim + 2;
    c->K = P->dim == 2 ? (4.0 - 2.0 * P->gamma) / (P->gamma - 1.0) : (3.0 - P->gamma) / (P->gamma - 1.0);
}

/* First-order fallback at a face point (a flagged option; the paper states
 * no limiter): a side whose reconstructed state has rho <= 0 or p <= 0 takes
 * avg, the average of the cell it was reconstructed from, with every
 * derivative zero.  Returns 1 when it applied. */
static int point_fallback(const Ctx *c, Side *S, const double *avg)
{
    int nv = c->nv;
    const double *q = S->D[0];
    double m2 = q[1] * q[1] + (nv == 4 ? q[2] * q[2] : 0.0);
    double p = (c->P->gamma - 1.0) * (q[nv - 1] - 0.5 * m2 / q[0]);
    if (q[0] > 0.0 && p > 0.0) return 0;
    for (int v = 0; v < nv; v++) {
        S->D[0][v] = avg[v];
        for (int k = 1; k < 6; k++) S->D[k][v] = 0.0;
    }
    return 1;
}

/* Build an ASE-DFF polynomial from a 1-D line of data. */
static int line_poly(const Ctx *c, const double q[5], const double qx[5], double h, const double sig[6], double P[9])
{
    double d[10];
    for (int k = 0; k < 5; k++) { d[k] = q[k]; d[5 + k] = h * qx[k]; }
    return ase_dff_poly(c, d, sig, P);
}

/* 1-D faces.  out: [5][3][nx+1]; sig: [nx+1]; branch: [nx+2] (cells -1..nx) */
int oracle_faces_1d(const OParams *P, const double *T, const double *W, const double *Wx,
                    const double *sx, const double *ghost, double dt,
                    double *out, double *sig, int *branch, int *nfall)
{
    Ctx c;
    ctx_init(&c, P, T, NULL, W, Wx, NULL, NULL, NULL, sx, NULL, ghost);
    int nx = P->nx, nv = 3, bad = 0;
    size_t nf = (size_t)nx + 1;
    /* Step 2 (the only step in 1-D): reconstruct cells -1..nx */
    double *fl = (double *)calloc((nx + 2) * 2 * 3 * 4, sizeof(double)); /* [cell][side][deriv][v] */
    for (int i = -1; i <= nx; i++) {
        double s4[6] = {sigx(&c, i - 2, 0), sigx(&c, i - 1, 0), sigx(&c, i, 0), sigx(&c, i + 1, 0), sigx(&c, i + 2, 0), sigx(&c, i + 3, 0)};
        for (int v = 0; v < nv; v++) {
            double q[5], qx[5], Pl[9];
            for (int k = 0; k < 5; k++) { q[k] = cellval(&c, K_W, v, 0, i + k - 2, 0); qx[k] = cellval(&c, K_WX, v, 0, i + k - 2, 0); }
            int b = line_poly(&c, q, qx, P->dx, s4, Pl);
            if (v == 0 && branch) branch[i + 1] = b;
            for (int s = 0; s < 2; s++) {
                double xi = s == 0 ? 0.5 : -0.5; /* s=0: right face (left state of i+1/2) */
                for (int nd = 0; nd < 3; nd++)
                    fl[(((size_t)(i + 1) * 2 + s) * 3 + nd) * 4 + v] = poly_der(Pl, xi, nd) / pow(P->dx, nd);
            }
        }
    }
    int nf_total = 0;
#pragma omp parallel for reduction(| : bad) reduction(+ : nf_total) schedule(static)
    for (int f = 0; f <= nx; f++) {
        Side L, R;
        memset(&L, 0, sizeof L); memset(&R, 0, sizeof R);
        int cl = f - 1, cr = f; /* left cell, right cell */
        for (int nd = 0; nd < 3; nd++)
            for (int v = 0; v < nv; v++) {
                L.D[nd][v] = fl[(((size_t)(cl + 1) * 2 + 0) * 3 + nd) * 4 + v];
                R.D[nd][v] = fl[(((size_t)(cr + 1) * 2 + 1) * 3 + nd) * 4 + v];
            }
        if (P->pt_fallback) {
            double al[3], ar[3];
            for (int v = 0; v < nv; v++) { al[v] = cellval(&c, K_W, v, 0, cl, 0); ar[v] = cellval(&c, K_W, v, 0, cr, 0); }
            nf_total += point_fallback(&c, &L, al) + point_fallback(&c, &R, ar);
        }
        double o[5][4];
        if (!kinetic_point(&c, &L, &R, dt, o)) bad = 1;
        for (int k = 0; k < 5; k++)
            for (int v = 0; v < nv; v++) out[((size_t)k * nv + v) * nf + f] = o[k][v];
        sig[f] = sigma_point(&c, L.D[0], R.D[0]);
    }
    free(fl);
    if (nfall) *nfall = nf_total;
    return bad ? FL_NONPHYS : 0;
}

/* 2-D faces of one direction.  dir 0: x-faces, out [5][4][ny][nx+1][m], sig [ny][nx+1][m];
 * dir 1: y-faces, out [5][4][ny+1][nx][m], sig [ny+1][nx][m].
 * branch (optional): per (cell, line) of the normal reconstruction, [ny+2][nx+2][m] for dir 0.
 * Results are in the global frame (rho, rhoU, rhoV, rhoE). */
int oracle_faces_2d(const OParams *P, const double *T, const double *gx, int dir,
                    const double *W, const double *Wx, const double *Wy, const double *Wxl,
                    const double *Wyl, const double *sx, const double *sy, double dt,
                    double *out, double *sig, int *nfall)
{
    Ctx c;
    ctx_init(&c, P, T, gx, W, Wx, Wy, Wxl, Wyl, sx, sy, NULL);
    const int nv = 4, m = P->m;
    /* work in (a, b) = (normal index, tangential index) */
    int na = dir == 0 ? P->nx : P->ny;  /* cells along the normal */
    int nb = dir == 0 ? P->ny : P->nx;  /* cells along the tangent */
    double hn = dir == 0 ? P->dx : P->dy, ht = dir == 0 ? P->dy : P->dx;
    int kW = K_W, kWn = dir == 0 ? K_WX : K_WY, kWt = dir == 0 ? K_WY : K_WX;
    int kLn = dir == 0 ? K_WXL : K_WYL;
    /* momentum components in the local frame: normal first */
    int vmap[4] = {0, dir == 0 ? 1 : 2, dir == 0 ? 2 : 1, 3};
#define CV(kind, v, l, a, b) (dir == 0 ? cellval(&c, kind, v, l, a, b) : cellval(&c, kind, v, l, b, a))
#define SN(f, b) (dir == 0 ? sigx(&c, f, b) : sigy(&c, b, f))  /* normal faces */
#define ST(a, g) (dir == 0 ? sigy(&c, a, g) : sigx(&c, g, a))  /* tangential faces of column a */

    /* Step 1: line averages along the normal direction at the m Gauss lines,
     * for cells a in [-3, na+2], b in [-1, nb]: tangential ASE-DFF. */
    int A0 = -3, NA = na + 6, B0 = -1, NB = nb + 2;
    double *la = (double *)malloc((size_t)NA * NB * m * nv * sizeof(double)); /* [b][a][l][v] local v */
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int bb = 0; bb < NB; bb++) {
        int b = B0 + bb;
        for (int aa = 0; aa < NA; aa++) {
            int a = A0 + aa;
            double s4[6] = {ST(a, b - 2), ST(a, b - 1), ST(a, b), ST(a, b + 1), ST(a, b + 2), ST(a, b + 3)};
            for (int v = 0; v < nv; v++) {
                int gv = vmap[v];
                double q[5], qt[5], Pt[9];
                for (int k = 0; k < 5; k++) { q[k] = CV(kW, gv, 0, a, b + k - 2); qt[k] = CV(kWt, gv, 0, a, b + k - 2); }
                line_poly(&c, q, qt, ht, s4, Pt);
                for (int l = 0; l < m; l++)
                    la[(((size_t)bb * NA + aa) * m + l) * nv + v] = poly_der(Pt, gx[l], 0);
            }
        }
    }
    /* Step 2: normal ASE-DFF on the line data, cells a in [-1, na], rows b in [-1, nb].
     * fr[b][a][side][l][deriv][v]: side 0 = value at the cell's +1/2 face, 1 = at its -1/2 face */
    int CA0 = -1, NCA = na + 2;
    double *fr = (double *)malloc((size_t)NB * NCA * 2 * m * 3 * nv * sizeof(double));
#define FR(bb, ca, s, l, nd, v) fr[(((((size_t)(bb) * NCA + (ca)) * 2 + (s)) * m + (l)) * 3 + (nd)) * nv + (v)]
#pragma omp parallel for schedule(static)
    for (int bb = 0; bb < NB; bb++) {
        int b = B0 + bb;
        for (int ca = 0; ca < NCA; ca++) {
            int a = CA0 + ca;
            double s4[6] = {SN(a - 2, b), SN(a - 1, b), SN(a, b), SN(a + 1, b), SN(a + 2, b), SN(a + 3, b)};
            for (int l = 0; l < m; l++)
                for (int v = 0; v < nv; v++) {
                    int gv = vmap[v];
                    double q[5], qn[5], Pn[9];
                    for (int k = 0; k < 5; k++) {
                        q[k] = la[(((size_t)bb * NA + (a + k - 2 - A0)) * m + l) * nv + v];
                        qn[k] = CV(kLn, gv, l, a + k - 2, b);
                    }
                    line_poly(&c, q, qn, hn, s4, Pn);
                    for (int s = 0; s < 2; s++)
                        for (int nd = 0; nd < 3; nd++)
                            FR(bb, ca, s, l, nd, v) = poly_der(Pn, s == 0 ? 0.5 : -0.5, nd) / pow(hn, nd);
                }
        }
    }
    /* Step 3 weights: nodes of the 3m face points of segments b-1, b, b+1 */
    double nodes[12], D1[4][12], D2[4][12];
    for (int s = 0; s < 3; s++)
        for (int l = 0; l < m; l++) nodes[s * m + l] = (s - 1) + gx[l];
    for (int l = 0; l < m; l++) {
        if (P->step3_deg == 0 || P->step3_deg >= 3 * m - 1) lagrange_der(nodes, 3 * m, gx[l], D1[l], D2[l]);
        else lsq_der(nodes, 3 * m, P->step3_deg, gx[l], D1[l], D2[l]);
    }

    /* faces f in [0, na] (face between cells f-1 and f), rows b in [0, nb) */
    size_t nf = (size_t)na + 1;
    int nf_total = 0;
#pragma omp parallel for reduction(| : bad) reduction(+ : nf_total) schedule(static)
    for (int b = 0; b < nb; b++) {
        int bb = b - B0;
        for (int f = 0; f <= na; f++) {
            for (int l = 0; l < m; l++) {
                Side S[2];
                memset(S, 0, sizeof S);
                for (int side = 0; side < 2; side++) {
                    /* left state: cell f-1 at its +1/2 face; right: cell f at its -1/2 face */
                    int a = side == 0 ? f - 1 : f;
                    int ca = a - CA0, sv = side == 0 ? 0 : 1;
                    /* tangential DFF: the r5 stencil of the reconstructing cell across
                     * the three face segments b-1, b, b+1 used by Step 3 */
                    double s6[6] = {ST(a, b - 2), ST(a, b - 1), ST(a, b), ST(a, b + 1), ST(a, b + 2), ST(a, b + 3)};
                    double Ast[6];
                    stencil_sums(P, s6, Ast);
                    double at = dff_alpha(Ast[ST_R5], P->sigma_thres);
                    for (int v = 0; v < nv; v++) {
                        S[side].D[0][v] = FR(bb, ca, sv, l, 0, v);
                        S[side].D[1][v] = FR(bb, ca, sv, l, 1, v);
                        S[side].D[2][v] = FR(bb, ca, sv, l, 2, v);
                        double wt = 0, wtt = 0, wnt = 0;
                        if (P->step3 == 0) {
                            for (int s = 0; s < 3; s++)
                                for (int k = 0; k < m; k++) {
                                    double w0 = FR(bb + s - 1, ca, sv, k, 0, v);
                                    double w1 = FR(bb + s - 1, ca, sv, k, 1, v);
                                    wt += D1[l][s * m + k] * w0;
                                    wtt += D2[l][s * m + k] * w0;
                                    wnt += D1[l][s * m + k] * w1;
                                }
                        } else {
                            double wm = FR(bb - 1, ca, sv, l, 0, v), w0 = FR(bb, ca, sv, l, 0, v), wp = FR(bb + 1, ca, sv, l, 0, v);
                            wt = 0.5 * (wp - wm);
                            wtt = wp - 2.0 * w0 + wm;
                            wnt = 0.5 * (FR(bb + 1, ca, sv, l, 1, v) - FR(bb - 1, ca, sv, l, 1, v));
                        }
                        S[side].D[3][v] = at * wt / ht;
                        S[side].D[4][v] = at * wtt / (ht * ht);
                        S[side].D[5][v] = at * wnt / ht;
                    }
                }
                if (P->pt_fallback)
                    for (int side = 0; side < 2; side++) {
                        double avg[4];
                        for (int v = 0; v < nv; v++) avg[v] = CV(kW, vmap[v], 0, side == 0 ? f - 1 : f, b);
                        nf_total += point_fallback(&c, &S[side], avg);
                    }
                double o[5][4];
                if (!kinetic_point(&c, &S[0], &S[1], dt, o)) bad = 1;
                /* out index: dir 0 -> [k][v][b][f][l] with b=j, f=i-face; dir 1 -> [k][v][f][b][l] */
                for (int k = 0; k < 5; k++)
                    for (int v = 0; v < nv; v++) {
                        size_t pos = dir == 0 ? ((((size_t)k * nv + vmap[v]) * nb + b) * nf + f) * m + l
                                              : ((((size_t)k * nv + vmap[v]) * nf + f) * nb + b) * m + l;
                        out[pos] = o[k][v];
                    }
                size_t ps = dir == 0 ? ((size_t)b * nf + f) * m + l : ((size_t)f * nb + b) * m + l;
                sig[ps] = sigma_point(&c, S[0].D[0], S[1].D[0]);
            }
        }
    }
    free(la);
    free(fr);
    if (nfall) *nfall = nf_total;
#undef CV
#undef SN
#undef ST
#undef FR
    return bad ? FL_NONPHYS : 0;
}

/* Exposed for the oracle's own pin tests: kinetic flux at a single point. */
int oracle_point_1d(const OParams *P, const double *D_l, const double *D_r, double dt, double *out)
{
    Ctx c;
    ctx_init(&c, P, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    Side L, R;
    memset(&L, 0, sizeof L); memset(&R, 0, sizeof R);
    for (int nd = 0; nd < 3; nd++)
        for (int v = 0; v < 3; v++) { L.D[nd][v] = D_l[nd * 3 + v]; R.D[nd][v] = D_r[nd * 3 + v]; }
    double o[5][4];
    int ok = kinetic_point(&c, &L, &R, dt, o);
    for (int k = 0; k < 5; k++)
        for (int v = 0; v < 3; v++) out[k * 3 + v] = o[k][v];
    return ok ? 0 : FL_NONPHYS;
}

/* 2-D point: D_l, D_r are [6][4] in the local frame (n = x). */
int oracle_point_2d(const OParams *P, const double *D_l, const double *D_r, double dt, double *out)
{
    Ctx c;
    ctx_init(&c, P, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    Side L, R;
    for (int nd = 0; nd < 6; nd++)
        for (int v = 0; v < 4; v++) { L.D[nd][v] = D_l[nd * 4 + v]; R.D[nd][v] = D_r[nd * 4 + v]; }
    double o[5][4];
    int ok = kinetic_point(&c, &L, &R, dt, o);
    for (int k = 0; k < 5; k++)
        for (int v = 0; v < 4; v++) out[k * 4 + v] = o[k][v];
    return ok ? 0 : FL_NONPHYS;
}

/* Maxwellian moments for the pin tests: mu[3][NMOM], mv[NMOM], mxi[4] */
int oracle_moments(const OParams *P, const double *W, double *mu, double *mv, double *mxi)
{
    Ctx c;
    ctx_init(&c, P, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    Maxw M;
    int ok = maxw_from_W(&c, W, &M);
    memcpy(mu, M.mu, sizeof M.mu);
    memcpy(mv, M.mv, sizeof M.mv);
    memcpy(mxi, M.mxi, sizeof M.mxi);
    return ok ? 0 : FL_NONPHYS;
}

/* micro-slope solve for the pin tests */
int oracle_micro_slope(const OParams *P, const double *W, const double *b, double *a)
{
    Ctx c;
    ctx_init(&c, P, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    Maxw M;
    int ok = maxw_from_W(&c, W, &M);
    micro_slope(&c, &M, b, a);
    return ok ? 0 : FL_NONPHYS;
}

/* Smoothness indicator of Eq. 3.13 for the pin tests (unit coordinate) */
double oracle_smoothness(const double *p, int deg)
{
    return smoothness(p, deg);
}

/* ASE-DFF polynomial of one cell for the pin tests */
int oracle_recon(const OParams *P, const double *T, const double *d, const double *sig6, double *poly)
{
    Ctx c;
    ctx_init(&c, P, T, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    return ase_dff_poly(&c, d, sig6, poly);
}
