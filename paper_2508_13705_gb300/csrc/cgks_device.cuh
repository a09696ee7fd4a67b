// Device code of the ASE-DFF compact gas-kinetic scheme (sm_103a).
//
// One stage of the S2O4 step (Sec. 2.2) runs as four kernels, each a
// grid-stride ("persistent") loop over the work items of every mesh in a
// descriptor table (one mesh, or a batch of uneven meshes):
//
//   k_lines   Sec. 3.3 Step 1: tangential ASE-DFF reconstruction of every cell
//             (plus a ghost halo), evaluated at the m Gauss lines of the
//             faces normal to x and to y -> line averages.
//   k_normal  Sec. 3.3 Step 2: normal ASE-DFF reconstruction of every
//             (cell, Gauss line) from line averages and line-averaged slopes
//             -> W, W_n, W_nn at the cell's two faces (Algorithm 1).
//   k_flux    Sec. 3.3 Step 3 (tangential W_t, W_tt, W_nt from the face values
//             of three face segments), Eq. 3.2 (sigma), Step 4 (kinetic
//             weighting, Eq. 2.7-2.8) and the time-integrated flux and
//             interface state of Eq. 2.6, 2.11, 2.12, 2.15 with the linear /
//             quadratic fits of Eq. 2.19-2.20 and 2.29 done analytically per
//             term; emits the per-point quantities the update needs.
//   k_update  Eq. 2.21-2.25, 2.30 and the Gauss-theorem slope update of
//             Sec. 3.3: cell averages, cell slopes and line slopes; the FP64
//             accumulator makes stage 2 need no stage-1 face data; face
//             sigma (Eq. 3.1) for the next step.
//
// Precision: R is the type of the reconstruction and kinetic arithmetic
// (double, or float for the FP32-bulk form).  Cell averages and their
// accumulation, the DFF (sigma, alpha, branch tests) and the positivity
// tests are always FP64.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tables.h"

namespace cgks {

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_FIXED = 2, BC_REFLECTIVE = 3, BC_NOSLIP = 4,
       BC_INFLOW = 5, BC_INFLOW_REFLECTIVE = 6 };
enum { ST_S0 = 0, ST_S1 = 1, ST_S2 = 2, ST_R5 = 3, ST_R7 = 4, ST_R9 = 5 };
enum { STATUS_NONPHYS = 1u };

struct TabF {
    float row[6][10][10];
    float cpoly[4][5][10];
    float bm2[3][3];
    float bm4[5][5];
    float gx[4], gw[4];
    float d1[4][12], d2[4][12];
};

static __constant__ CgksTables c_tab[3];  // orders 5, 7, 9 (one copy per translation unit)
static __constant__ TabF c_tabf[3];

template <typename R> struct Tab;
template <> struct Tab<double> {
    __device__ static const CgksTables& get(int oi) { return c_tab[oi]; }
};
template <> struct Tab<float> {
    __device__ static const TabF& get(int oi) { return c_tabf[oi]; }
};

// Per-mesh descriptor (device memory); a batch is an array of these.
struct Mesh {
    int nx, ny, order, oi;          // oi: 0, 1, 2 for orders 5, 7, 9
    int bc[4];
    int tau_mode;
    int dff_lag;                    // 0: sigma of step n-1; 1: stage 2 uses stage 1's
    int pf;                         // first-order fallback at non-physical face points
    double dx, dy, gamma, K, thr, ghi, glo, eps, c1, c2, cfl;
    double idx, idy;                // 1 / dx, 1 / dy
    double mu;                      // dynamic viscosity (tau_mode 2)
    double x0, y0;                  // lower-left corner
    double bcs[4][2][4];            // inflow ghost states per side: [0] below the split, [1] beyond
    double bcx[4][2];               // split point along the side: bcx[0] + bcx[1] t
    float muf;
    float gf, Kf, c1f, c2f, idxf, idyf;  // FP32-bulk copies (no per-point conversions)
    float idxlo, idylo;             // low parts: idx = idxf + idxlo to float-float accuracy
    long long plane;                // nx * ny
    // state: planes of nx*ny doubles.  2-D: W[4] Wx[4] Wy[4] Wxl[m][4] Wyl[m][4];
    // 1-D: W[3] Wx[3]
    double *S0, *S1;                // S0: state n (and n+1), S1: stage-1 state W*
    float *F0, *F1;                 // FP32-bulk form: float copies of all planes of S0 / S1,
                                    // then the low parts float(W - float(W)) of the cell
                                    // averages (the FP64 planes hold the cell averages;
                                    // their slope planes are rebuilt from these on read-out)
    double *ACC;                    // 2-D: W[4] Wxl[m][4] Wyl[m][4]; 1-D: W[3] Wface[3]
    double *sig_x, *sig_y;          // sigma of the previous step [ny][nx+1], [ny+1][nx]
    double *sig_xn, *sig_yn;        // sigma being built this step
    const double* ghost;            // 1-D fixed BC ghost cells
    void *FR[2], *FO[2];            // scratch per direction (R typed)
    void* AT[2];                    // tangential r5 DFF per cell (R typed)
    void* TD[2];                    // FP32 bulk: hi(a, b-1) - hi(a, b), hi(a, b+1) - hi(a, b)
                                    // of each cell, local frame, [8] floats
    double* SP[2];                  // sigma per face Gauss point
    double* dt;                     // device scalar (this mesh's step)
    float* dtf;                     // the same in FP32: [0] float(dt), [1] float(dt - [0])
    double* t;                      // device scalar (simulated time)
    double* tn;                     // device scalar: t^n of the step in flight
    unsigned long long* nfall;      // face-point sides that took the fallback
    unsigned* status;
    long long* bad;
    unsigned long long* smax;       // CFL reduction (bits of a positive double)
    unsigned long long* branch;     // [4] AO, r5, r7, r9 counts
};

// Prefix sums of the work items of every kernel over the meshes of a table,
// and the first mesh's descriptor by value: a launch over one mesh reads its
// descriptor from the kernel parameters (constant-bank operands) instead of
// loading it from the table in every grid-stride iteration.
struct Work {
    const Mesh* mesh;
    const long long* off;  // [n+1] prefix of items
    int n;
    long long total;
    Mesh m0;               // mesh[0]
};

__device__ __forceinline__ int find_mesh(const Work& w, long long g)
{
    int lo = 0, hi = w.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (w.off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The mesh of work item gi and the item's index within it.  ONE: the launch
// covers a single mesh (offset 0), taken from the parameters.
template <bool ONE>
__device__ __forceinline__ const Mesh& mesh_of(const Work& w, long long gi, long long& local)
{
    if (ONE) { local = gi; return w.m0; }
    const int k = find_mesh(w, gi);
    local = gi - w.off[k];
    return w.mesh[k];
}

__device__ __forceinline__ int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

// ------------------------------------------------------------------ ghost cells

// Mesh constants in the bulk precision R.
template <typename R> struct MeshR;
template <> struct MeshR<double> {
    __device__ static double gamma(const Mesh& g) { return g.gamma; }
    __device__ static double K(const Mesh& g) { return g.K; }
    __device__ static double c1(const Mesh& g) { return g.c1; }
    __device__ static double c2(const Mesh& g) { return g.c2; }
    __device__ static double mu(const Mesh& g) { return g.mu; }
    __device__ static double ih(const Mesh& g, int dir) { return dir == 0 ? g.idx : g.idy; }
    __device__ static double dt(const Mesh& g) { return *g.dt; }
};
template <> struct MeshR<float> {
    __device__ static float gamma(const Mesh& g) { return g.gf; }
    __device__ static float K(const Mesh& g) { return g.Kf; }
    __device__ static float c1(const Mesh& g) { return g.c1f; }
    __device__ static float c2(const Mesh& g) { return g.c2f; }
    __device__ static float mu(const Mesh& g) { return g.muf; }
    __device__ static float ih(const Mesh& g, int dir) { return dir == 0 ? g.idxf : g.idyf; }
    __device__ static float dt(const Mesh& g) { return *g.dtf; }
};

// The state planes the bulk arithmetic reads: FP64 planes for R = double,
// the float copies for R = float.  which: 0 state n, 1 stage-1 state.
template <typename R> __device__ __forceinline__ const R* state_planes(const Mesh& g, int which);
template <> __device__ __forceinline__ const double* state_planes<double>(const Mesh& g, int which)
{
    return which == 0 ? g.S0 : g.S1;
}
template <> __device__ __forceinline__ const float* state_planes<float>(const Mesh& g, int which)
{
    return which == 0 ? g.F0 : g.F1;
}

__device__ __forceinline__ bool is_wall(int bc) { return bc == BC_REFLECTIVE || bc == BC_NOSLIP; }
// sides whose ghost faces mirror sigma (a wall along all or part of the side)
__device__ __forceinline__ bool is_mirror(int bc) { return is_wall(bc) || bc == BC_INFLOW_REFLECTIVE; }

// Time at which a stage takes prescribed ghost states: t^n in stage 1, the
// stage-2 state lives at t^n + dt/2.
__device__ __forceinline__ double stage_time(const Mesh& g, int stage)
{
    return stage == 1 ? *g.tn : *g.tn + 0.5 * *g.dt;
}

// Inflow sides: is the centre of ghost row / column k, along side `side`
// (y on the x-sides, x on the y-sides), below the split point at time tb?
__device__ __forceinline__ bool below_split(const Mesh& g, int side, int k, double tb)
{
    double s = side < 2 ? g.y0 + (k + 0.5) * g.dy : g.x0 + (k + 0.5) * g.dx;
    return s < g.bcx[side][0] + g.bcx[side][1] * tb;
}

// Sign of a ghost value mirrored across a wall with normal x (normal = 0) or
// y (normal = 1): reflection maps q to S q(-x), S reversing the normal
// momentum (slip wall) or every momentum component (no-slip wall); a
// derivative along the normal takes one more sign.
template <int D>
__device__ __forceinline__ bool wall_flip(int kind, int v, int normal, int bc)
{
    bool rev = (v == 1 + normal) || (bc == BC_NOSLIP && v >= 1 && v <= D);
    bool dnormal = normal == 0 ? (kind == 1 || kind == 3) : (kind == 2 || kind == 4);
    return rev != dnormal;
}

// The low part of a cell average in the FP32-bulk form: the FP64 average x is
// held as hi = float(x) (the W planes) plus lo = float(x - hi) (the planes
// after all others); FP64 planes need no low part.
template <typename T> __device__ __forceinline__ T low_part(double x) { return (T)(x - (double)(T)x); }
template <> __device__ __forceinline__ double low_part<double>(double) { return 0.0; }

// A prescribed ghost value x (fixed ghost cells, inflow states) as kind asks:
// the value (kind 0), its low part (kind 5), or a zero slope.
template <typename T> __device__ __forceinline__ T prescribed(double x, int kind)
{
    return kind == 0 ? (T)x : (kind == 5 ? low_part<T>(x) : (T)0);
}

// kind: 0 W, 1 Wx, 2 Wy, 3 Wx_line, 4 Wy_line (global orientation), 5 the low
// part of W (FP32-bulk float planes only); tb: the
// stage's time, read by inflow sides only.  Ghost rules apply x first, then y.
// WALLS = false compiles the wall and inflow branches out: the stencil kernels
// have an instance for meshes without them, whose hot loops the (never
// taken) code would otherwise slow down.
template <int D, int M, typename T, bool WALLS = true>
__device__ __forceinline__ T cell(const Mesh& g, const T* S, int kind, int v, int l, int i, int j, double tb)
{
    bool zero = false, neg = false;
    if (i < 0 || i >= g.nx) {
        int side = i < 0 ? 0 : 1;
        int bc = g.bc[side];
        if (bc == BC_PERIODIC) {
            i = imod(i, g.nx);
        } else if (bc == BC_FIXED) {
            int layer = side == 0 ? (-1 - i) : (i - g.nx);
            double gv = g.ghost[((side * 3 + layer) * 2 + (kind == 0 || kind == 5 ? 0 : 1)) * 3 + v];
            return kind == 5 ? low_part<T>(gv) : (T)gv;
        } else if (WALLS && (bc == BC_INFLOW || (bc == BC_INFLOW_REFLECTIVE && below_split(g, side, j, tb)))) {
            // prescribed state by the row's centre, zero slopes
            return prescribed<T>(g.bcs[side][below_split(g, side, j, tb) ? 0 : 1][v], kind);
        } else if (WALLS && is_mirror(bc)) {
            // ghost cell -1-k mirrors cell k; lines across x (Wy_line) swap ends
            i = i < 0 ? -1 - i : 2 * g.nx - 1 - i;
            neg = wall_flip<D>(kind, v, 0, bc);
            if (kind == 4) l = M - 1 - l;
        } else {
            i = i < 0 ? 0 : g.nx - 1;
            zero = (kind == 1 || kind == 3);
        }
    }
    if (D == 2 && (j < 0 || j >= g.ny)) {
        int side = j < 0 ? 2 : 3;
        int bc = g.bc[side];
        if (WALLS && (bc == BC_INFLOW || (bc == BC_INFLOW_REFLECTIVE && below_split(g, side, i, tb)))) {
            // prescribed state by the column's centre (after the x rule), zero slopes
            T val = prescribed<T>(g.bcs[side][below_split(g, side, i, tb) ? 0 : 1][v], kind);
            return neg ? -val : val;
        }
        if (bc == BC_PERIODIC) {
            j = imod(j, g.ny);
        } else if (WALLS && is_mirror(bc)) {
            j = j < 0 ? -1 - j : 2 * g.ny - 1 - j;
            neg = neg != wall_flip<D>(kind, v, 1, bc);
            if (kind == 3) l = M - 1 - l;
        } else {
            j = j < 0 ? 0 : g.ny - 1;
            zero = zero || (kind == 2 || kind == 4);
        }
    }
    if (zero) return (T)0;
    long long idx = (long long)j * g.nx + i;
    int p;
    if (D == 1) {
        p = kind == 0 ? v : (kind == 5 ? 6 + v : 3 + v);
    } else {
        switch (kind) {
        case 0: p = v; break;
        case 1: p = 4 + v; break;
        case 2: p = 8 + v; break;
        case 3: p = 12 + 4 * l + v; break;
        case 5: p = 12 + 8 * M + v; break;
        default: p = 12 + 4 * M + 4 * l + v; break;
        }
    }
    T val = S[p * g.plane + idx];
    return neg ? -val : val;
}

// sigma of x-face f (between cells f-1 and f) in row j; ghost faces: periodic
// wrap, otherwise 0 beyond the boundary face and the nearest row across y.
template <int D, bool WALLS = true>
__device__ __forceinline__ double sigx(const Mesh& g, const double* sx, int f, int j)
{
    if (f < 0 || f > g.nx) {
        int bc = g.bc[f < 0 ? 0 : 1];
        if (bc == BC_PERIODIC) f = imod(f, g.nx);
        else if (WALLS && is_mirror(bc)) f = f < 0 ? -f : 2 * g.nx - f;  // beyond a wall: the mirrored face
        else return 0.0;
    }
    if (D == 2 && (j < 0 || j >= g.ny)) {
        int bc = g.bc[j < 0 ? 2 : 3];
        if (bc == BC_PERIODIC) j = imod(j, g.ny);
        else if (WALLS && is_mirror(bc)) j = j < 0 ? -1 - j : 2 * g.ny - 1 - j;
        else j = j < 0 ? 0 : g.ny - 1;
    }
    return sx[(long long)j * (g.nx + 1) + f];
}

template <bool WALLS = true>
__device__ __forceinline__ double sigy(const Mesh& g, const double* sy, int i, int f)
{
    if (f < 0 || f > g.ny) {
        int bc = g.bc[f < 0 ? 2 : 3];
        if (bc == BC_PERIODIC) f = imod(f, g.ny);
        else if (WALLS && is_mirror(bc)) f = f < 0 ? -f : 2 * g.ny - f;
        else return 0.0;
    }
    if (i < 0 || i >= g.nx) {
        int bc = g.bc[i < 0 ? 0 : 1];
        if (bc == BC_PERIODIC) i = imod(i, g.nx);
        else if (WALLS && is_mirror(bc)) i = i < 0 ? -1 - i : 2 * g.nx - 1 - i;
        else i = i < 0 ? 0 : g.nx - 1;
    }
    return sy[(long long)f * g.nx + i];
}

// 16-byte vector moves of 4 consecutive values (float4, or two double2)
__device__ __forceinline__ void ld4(const float* p, float v[4])
{
    float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4])
{
    double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4])
{
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// ------------------------------------------------------------------ float-float
// Unevaluated sums hi + lo of two floats (Dekker's double-length arithmetic,
// with Knuth's two-sum and the FMA two-product), about 44 significant bits:
// FP64-level accuracy from FP32 instructions, for the few O(1) quantities of
// the FP32-bulk form whose rounding would otherwise enter every update.  The
// explicit _rn intrinsics keep the compiler from contracting or reassociating.
struct ff { float hi, lo; };

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff ff_norm(float hi, float lo)  // |hi| >= |lo|
{
    float s = __fadd_rn(hi, lo);
    return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.hi, b.hi);
    return ff_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return ff_norm(p, e);
}
__device__ __forceinline__ ff ff_of(float a) { return {a, 0.0f}; }
// a / b of two floats: the remainder a - q b of the rounded quotient is exact
__device__ __forceinline__ ff ff_div(float a, float b)
{
    float q = __fdiv_rn(a, b);
    return ff_norm(q, __fdiv_rn(__fmaf_rn(-q, b, a), b));
}
__device__ __forceinline__ double ff_val(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// Euler flux along the local normal of a state given by floats (rho, m_n,
// m_t, E) (2-D, D = 2) or (rho, m, E) (1-D), in float-float: (m_n, m_n u + p,
// m_t u, u (E + p)) with u = m_n / rho, p = (gamma - 1)(E - (m_n u + m_t v) / 2).
// gm1 = gamma - 1 as a float-float.
template <int D>
__device__ __forceinline__ void euler_flux_ff(const float* w, ff gm1, ff* F)
{
    const float rho = w[0], mn = w[1], mt = D == 2 ? w[2] : 0.0f, E = w[D + 1];
    ff u = ff_div(mn, rho);
    ff v = ff_div(mt, rho);
    ff ke = ff_add(ff_mul(ff_of(mn), u), ff_mul(ff_of(mt), v));  // rho |U|^2
    ff p = ff_mul(gm1, ff_add(ff_of(E), ff_mul(ff_of(-0.5f), ke)));
    F[0] = ff_of(mn);
    F[1] = ff_add(ff_mul(ff_of(mn), u), p);
    if (D == 2) F[2] = ff_mul(ff_of(mt), u);
    F[D + 1] = ff_mul(u, ff_add(ff_of(E), p));
}

// F(w0 + q) - F(w0) of the Euler flux along the local normal, by algebra in
// which every term is a product with a component of q (no difference of two
// O(1) values), so the result keeps the relative accuracy of q.  w0: the base
// state (floats), q: the increment; same layouts as euler_flux_ff.
template <int D, typename R>
__device__ __forceinline__ void euler_flux_delta(const R* w0, const R* q, R gm1, R* dF)
{
    const R r0 = w0[0], mn0 = w0[1], mt0 = D == 2 ? w0[2] : (R)0, E0 = w0[D + 1];
    const R dr = q[0], dmn = q[1], dmt = D == 2 ? q[2] : (R)0, dE = q[D + 1];
    const R ir0 = (R)1 / r0;
    const R u0 = mn0 * ir0, v0 = mt0 * ir0;
    const R ir = (R)1 / (r0 + dr);
    const R du = (dmn - u0 * dr) * ir, dv = (dmt - v0 * dr) * ir;  // u - u0, v - v0
    const R u = u0 + du;
    // kinetic energy rho |U|^2 / 2: its change, product by product
    const R dke = (R)0.5 * (dr * (u0 * u0 + v0 * v0) + (r0 + dr) * (du * ((R)2 * u0 + du) + dv * ((R)2 * v0 + dv)));
    const R p0 = gm1 * (E0 - (R)0.5 * r0 * (u0 * u0 + v0 * v0));
    const R dp = gm1 * (dE - dke);
    dF[0] = dmn;
    dF[1] = dmn * u + mn0 * du + dp;             // (m u + p) - (m0 u0 + p0)
    if (D == 2) dF[2] = dmt * u + mt0 * du;      // m_t u - m_t0 u0
    dF[D + 1] = du * (E0 + p0) + u * (dE + dp);  // u H - u0 H0, H = E + p
}

// ------------------------------------------------------------------ ASE-DFF

// Branch and stencil DFFs of one cell from the sigma of the six faces
// i-5/2 .. i+5/2 (Eq. 3.3-3.4).  A stencil's sum covers every face of every
// cell it draws data from; eta = 2 for r9.  Algorithm 1 picks the branch.
struct Dff {
    double a[4];   // alpha of S0, S1, S2, r5
    double alpha;  // alpha of the linear stencil used
    int st;        // linear stencil, or -1 for HWENO-AO
};

__device__ __forceinline__ double dff_alpha(double A, double thr) { return A < thr ? 1.0 : thr / A; }

__device__ __forceinline__ Dff dff_select(int order, const double s[6], double thr)
{
    // The threshold tests come first; a DFF below 1 (a division) is formed
    // only on the HWENO-AO branch, where the sub-stencil DFFs are used.  On
    // every linear branch the chosen stencil's DFF is 1 by construction.
    Dff d;
    double A_r5 = s[1] + s[2] + s[3] + s[4];
    double A_r7 = s[0] + A_r5 + s[5];
    d.a[0] = d.a[1] = d.a[2] = d.a[3] = 1.0;
    d.alpha = 1.0;
    if (A_r5 >= thr) {
        d.st = -1;
        d.a[0] = dff_alpha(s[1] + s[2] + s[3], thr);
        d.a[1] = dff_alpha(s[2] + s[3] + s[4], thr);
        d.a[2] = d.a[3] = d.alpha = thr / A_r5;
    } else if (order == 5 || A_r7 >= thr) {
        d.st = ST_R5;
    } else if (order == 7 || 2.0 * A_r7 >= thr) {
        d.st = ST_R7;
    } else {
        d.st = ST_R9;
    }
    return d;
}

// A cell's DFF choice in the bulk precision R: the DFFs of S0, S1, S2 = r5
// (a[2] == a[3]) and the stencil code (-1 HWENO-AO, else r5/r7/r9).  On the
// linear branches the chosen stencil's DFF is 1 (Algorithm 1 only takes a
// linear stencil whose DFF is 1), so only the HWENO-AO branch scales.
template <typename R>
struct DffR {
    R a[4];
    int st;
};

template <typename R>
__device__ __forceinline__ DffR<R> dff_r(const Dff& d)
{
    DffR<R> r;
    for (int k = 0; k < 4; ++k) r.a[k] = (R)d.a[k];
    r.st = d.st;
    return r;
}

// Packed form for a per-cell buffer: (a0, a1, a3, stencil code)
template <typename R>
__device__ __forceinline__ void dff_pack(const DffR<R>& d, R out[4])
{
    out[0] = d.a[0]; out[1] = d.a[1]; out[2] = d.a[3]; out[3] = (R)d.st;
}
template <typename R>
__device__ __forceinline__ DffR<R> dff_unpack(const R in[4])
{
    DffR<R> d;
    d.a[0] = in[0]; d.a[1] = in[1]; d.a[2] = d.a[3] = in[2];
    d.st = (int)in[3];
    return d;
}

// HWENO-AO(5,3) with DFF-scaled sub-polynomials (Eq. 3.11-3.17, 3.19) for
// NOUT consecutive functional rows starting at row0.  Kept out of line: the
// branch is rare, and inlining it in every variable's loop bloats the kernels.
template <typename R, int NOUT>
__device__ __noinline__ void recon_ao(const R* al, int oi, int row0, const R* dp, R* out, R ghi, R glo, R eps)
{
    const auto& T = Tab<R>::get(oi);
    R beta[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        R c[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) {
            R s = 0;
#pragma unroll
            for (int q = 0; q < 10; ++q) s += T.cpoly[k][n][q] * dp[q];
            c[n] = s;
        }
        R b = 0;
        if (k < 3) {
#pragma unroll
            for (int x = 1; x < 3; ++x)
#pragma unroll
                for (int y = 1; y < 3; ++y) b += c[x] * c[y] * T.bm2[x][y];
        } else {
#pragma unroll
            for (int x = 1; x < 5; ++x)
#pragma unroll
                for (int y = 1; y < 5; ++y) b += c[x] * c[y] * T.bm4[x][y];
        }
        beta[k] = al[k] * al[k] * b;  // smoothness of the DFF-scaled polynomial
    }
    R g3 = ghi, g2 = ((R)1 - ghi) * glo, g0 = ((R)1 - ghi) * ((R)1 - glo) * (R)0.5;
    R gk[4] = {g0, g0, g2, g3};
    R tz = (fabs(beta[3] - beta[0]) + fabs(beta[3] - beta[1]) + fabs(beta[3] - beta[2])) / (R)3;
    R w[4], ws = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        R q = tz / (beta[k] + eps);
        w[k] = gk[k] * ((R)1 + q * q);
        ws += w[k];
    }
    R inv = (R)1 / ws;
    R c3 = w[3] * inv / g3;
    R ck[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ck[k] = w[k] * inv - w[3] * inv * gk[k] / g3;
#pragma unroll
    for (int r = 0; r < NOUT; ++r) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            R p = 0;
#pragma unroll
            for (int q = 0; q < 10; ++q) p += T.row[k][row0 + r][q] * dp[q];
            s += (k == 3 ? c3 : ck[k]) * al[k] * p;
        }
        out[r] = s;
    }
}

// Evaluate NOUT consecutive functional rows (from row0) of the ASE-DFF
// polynomial of one cell.  dp[10]: data relative to the own cell:
// [Qbar_{i+k} - Qbar_i (k=-2..2), h*Qx_{i+k}]; values come out relative to
// Qbar_i too (Eq. 3.5: Q_i + alpha (p - Q_i), derivatives alpha p').
template <typename R, int NOUT>
__device__ __forceinline__ void recon(const DffR<R>& dff, int oi, int row0, const R dp[10], R out[NOUT],
                                      R ghi, R glo, R eps)
{
    if (dff.st >= 0) {
        const auto& T = Tab<R>::get(oi);
#pragma unroll
        for (int r = 0; r < NOUT; ++r) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < 10; ++k) s += T.row[dff.st][row0 + r][k] * dp[k];
            out[r] = s;
        }
        return;
    }
    recon_ao<R, NOUT>(dff.a, oi, row0, dp, out, ghi, glo, eps);
}

// The taps of dp = (Qbar_{i-2..i+2} - Qbar_i, h Qx_{i-2..i+2}) that a linear
// stencil of Sec. 3.2 uses: the own average enters only through the
// differences (dp[2] = 0) and the own gradient not at all; r5 spans cells
// i-1..i+1 with the neighbour gradients, r7 cells i-2..i+2 with the gradients
// of i-1 and i+1, r9 cells i-2..i+2 with the four neighbour gradients.
__host__ __device__ constexpr bool st_tap(int st, int k)
{
    return st == ST_R9 ? (k != 2 && k != 7)
         : st == ST_R7 ? (k == 0 || k == 1 || k == 3 || k == 4 || k == 6 || k == 8)
         : st == ST_R5 ? (k == 1 || k == 3 || k == 6 || k == 8)
         : true;
}

// A linear stencil with the order (table index OI), the stencil and the first
// output row fixed at compile time, for the 2-D kernels, whose instantiation
// fixes the order: the stencil row comes from a constant address, so the
// coefficients enter the FMAs as constant-bank operands instead of loads.
template <typename R, int NOUT, int OI, int ST, int ROW0>
__device__ __forceinline__ void recon_lin(const R dp[10], R out[NOUT])
{
    const auto& T = Tab<R>::get(OI);
#pragma unroll
    for (int r = 0; r < NOUT; ++r) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < 10; ++k)
            if (st_tap(ST, k)) s += T.row[ST][ROW0 + r][k] * dp[k];
        out[r] = s;
    }
}

// Compile-time stencil tag (-1: HWENO-AO) for branch-hoisted reconstruction
// loops: the branch on a cell's stencil is taken once, outside the loop over
// variables, so each branch is one straight run of code.
template <int V> struct StTag { static constexpr int value = V; };

// Reconstruction with the stencil fixed at compile time (ST = -1: HWENO-AO).
template <typename R, int NOUT, int OI, int ST, int ROW0>
__device__ __forceinline__ void recon_st(const DffR<R>& dff, const R dp[10], R out[NOUT], R ghi, R glo, R eps)
{
    if constexpr (ST >= 0) recon_lin<R, NOUT, OI, ST, ROW0>(dp, out);
    else recon_ao<R, NOUT>(dff.a, OI, ROW0, dp, out, ghi, glo, eps);
}

// Calls body(StTag<st>()) for the stencil of dff; the order (table index OI)
// bounds the linear stencils that can occur.
template <int OI, typename R, typename Body>
__device__ __forceinline__ void with_stencil(const DffR<R>& dff, Body&& body)
{
    if (OI == 2 && dff.st == ST_R9) body(StTag<(OI == 2 ? ST_R9 : ST_R5)>());
    else if (OI >= 1 && dff.st == ST_R7) body(StTag<(OI >= 1 ? ST_R7 : ST_R5)>());
    else if (dff.st == ST_R5) body(StTag<ST_R5>());
    else body(StTag<-1>());
}


// ------------------------------------------------------------------ kinetics

// Maxwellian moments per unit density for one velocity range, with the
// per-state factors the micro-slope solves reuse (1/rho, 1/(2 lambda),
// 4 lambda^2 / (K + D), U^2 + V^2 + (K + D) / (2 lambda)).
template <typename R, int D>
struct Mom {
    R rho, U, V, lam;
    R ir, il, c4, cs;
    R mu[7];
    R mv[6];
    R x2, x4;
};

// range: 0 full, 1 u > 0, 2 u < 0.  Returns false if rho or p <= 0.
template <typename R, int D>
__device__ __forceinline__ bool maxwellian(const R* W, R gamma, R K, int range, Mom<R, D>& M)
{
    R rho = W[0];
    R ir = (R)1 / rho;
    R U = W[1] * ir;
    R V = D == 2 ? W[2] * ir : (R)0;
    R p = (gamma - (R)1) * (W[D + 1] - (R)0.5 * rho * (U * U + V * V));
    R lam = (R)0.5 * rho / p;
    R i2l = p * ir;  // 1 / (2 lambda)
    M.rho = rho; M.U = U; M.V = V; M.lam = lam;
    M.ir = ir; M.il = i2l;
    M.c4 = (R)4 * lam * lam / (K + (R)D);
    M.cs = U * U + V * V + (K + (R)D) * i2l;
    if (range == 0) {
        M.mu[0] = 1; M.mu[1] = U;
    } else {
        R sl = sqrt(lam);
        R e = exp(-lam * U * U) * (R)0.28209479177387814 * rsqrt(lam);  // e^{-lam U^2} / (2 sqrt(pi lam))
        if (range == 1) { M.mu[0] = (R)0.5 * erfc(-sl * U); M.mu[1] = U * M.mu[0] + e; }
        else { M.mu[0] = (R)0.5 * erfc(sl * U); M.mu[1] = U * M.mu[0] - e; }
    }
#pragma unroll
    for (int n = 0; n < 5; ++n) M.mu[n + 2] = U * M.mu[n + 1] + (R)(n + 1) * i2l * M.mu[n];
    if (D == 2) {
        M.mv[0] = 1; M.mv[1] = V;
#pragma unroll
        for (int n = 0; n < 4; ++n) M.mv[n + 2] = V * M.mv[n + 1] + (R)(n + 1) * i2l * M.mv[n];
    }
    M.x2 = K * i2l;
    M.x4 = K * (K + (R)2) * i2l * i2l;
    return rho > (R)0 && p > (R)0;
}

// <a u^p v^q psi> per unit density, a = (a1, a2, a3, a4) on psi =
// (1, u, v, (u^2+v^2+xi^2)/2) [2-D] or a = (a1, a2, a3) on (1, u, (u^2+xi^2)/2).
template <typename R, int D>
__device__ __forceinline__ void mom(const Mom<R, D>& M, const R* a, int p, int q, R* out)
{
    if (D == 2) {
        auto A = [&](int i, int j, bool xs) -> R {
            R x0 = xs ? M.x2 : (R)1, x1 = xs ? M.x4 : M.x2;
            R base = a[0] * M.mu[i] * M.mv[j] + a[1] * M.mu[i + 1] * M.mv[j] + a[2] * M.mu[i] * M.mv[j + 1]
                   + (R)0.5 * a[3] * (M.mu[i + 2] * M.mv[j] + M.mu[i] * M.mv[j + 2]);
            return x0 * base + (R)0.5 * a[3] * x1 * M.mu[i] * M.mv[j];
        };
        out[0] = A(p, q, false);
        out[1] = A(p + 1, q, false);
        out[2] = A(p, q + 1, false);
        out[3] = (R)0.5 * (A(p + 2, q, false) + A(p, q + 2, false) + A(p, q, true));
    } else {
        auto A = [&](int i, bool xs) -> R {
            R x0 = xs ? M.x2 : (R)1, x1 = xs ? M.x4 : M.x2;
            return x0 * (a[0] * M.mu[i] + a[1] * M.mu[i + 1] + (R)0.5 * a[2] * M.mu[i + 2])
                 + (R)0.5 * a[2] * x1 * M.mu[i];
        };
        out[0] = A(p, false);
        out[1] = A(p + 1, false);
        out[2] = (R)0.5 * (A(p + 2, false) + A(p, true));
    }
}

// Closed-form solution of <a> = b (full-range moments, Eq. 2.8), using the
// per-state factors of the Maxwellian.
template <typename R, int D>
__device__ __forceinline__ void slope(const Mom<R, D>& M, R K, const R* b, R* a)
{
    (void)K;
    if (D == 2) {
        R B0 = b[0] * M.ir, B1 = b[1] * M.ir, B2 = b[2] * M.ir, B3 = b[3] * M.ir;
        R R2 = B1 - M.U * B0, R3 = B2 - M.V * B0;
        R R4 = (R)2 * B3 - M.cs * B0;
        R a4 = M.c4 * (R4 - (R)2 * M.U * R2 - (R)2 * M.V * R3);
        R a3 = (R)2 * M.lam * R3 - M.V * a4;
        R a2 = (R)2 * M.lam * R2 - M.U * a4;
        a[0] = B0 - M.U * a2 - M.V * a3 - (R)0.5 * a4 * M.cs;
        a[1] = a2; a[2] = a3; a[3] = a4;
    } else {
        R B0 = b[0] * M.ir, B1 = b[1] * M.ir, B2 = b[2] * M.ir;
        R R2 = B1 - M.U * B0;
        R R3 = (R)2 * B2 - M.cs * B0;
        R a3 = M.c4 * (R3 - (R)2 * M.U * R2);
        R a2 = (R)2 * M.lam * R2 - M.U * a3;
        a[0] = B0 - M.U * a2 - (R)0.5 * a3 * M.cs;
        a[1] = a2; a[2] = a3;
    }
}

// Moments linear in the micro-slope: <a u^p v^q psi> = sum_k a_k G[k][i] with
// the symmetric Gram matrix G[k][i] = <u^p v^q psi_k psi_i> per unit density.
// A matrix serves every product with the same (p, q) and Maxwellian, which
// costs a 4 x 4 multiply instead of a moment expansion each.  Stored as the
// upper triangle: 2-D (00 01 02 03 11 12 13 22 23 33), 1-D (00 01 02 11 12 22).
template <typename R, int D>
struct Gram { R g[D == 2 ? 10 : 6]; };

template <typename R, int D, int P, int Q>
__device__ __forceinline__ void gram(const Mom<R, D>& M, Gram<R, D>& G)
{
    const R* m = M.mu + P;
    if (D == 2) {
        const R* v = M.mv + Q;
        G.g[0] = m[0] * v[0];
        G.g[1] = m[1] * v[0];
        G.g[2] = m[0] * v[1];
        G.g[3] = (R)0.5 * (m[2] * v[0] + m[0] * v[2] + M.x2 * G.g[0]);
        G.g[4] = m[2] * v[0];
        G.g[5] = m[1] * v[1];
        G.g[6] = (R)0.5 * (m[3] * v[0] + m[1] * v[2] + M.x2 * G.g[1]);
        G.g[7] = m[0] * v[2];
        G.g[8] = (R)0.5 * (m[2] * v[1] + m[0] * v[3] + M.x2 * G.g[2]);
        G.g[9] = (R)0.25 * (m[4] * v[0] + m[0] * v[4] + M.x4 * G.g[0]
                            + (R)2 * (m[2] * v[2] + M.x2 * (G.g[4] + G.g[7])));
    } else {
        G.g[0] = m[0];
        G.g[1] = m[1];
        G.g[2] = (R)0.5 * (m[2] + M.x2 * m[0]);
        G.g[3] = m[2];
        G.g[4] = (R)0.5 * (m[3] + M.x2 * m[1]);
        G.g[5] = (R)0.25 * (m[4] + (R)2 * M.x2 * m[2] + M.x4 * m[0]);
    }
}

// out_i = s * sum_k a_k G[k][i]
template <typename R, int D>
__device__ __forceinline__ void gmul(const Gram<R, D>& G, const R* a, R s, R* out)
{
    if (D == 2) {
        const R* g = G.g;
        out[0] = s * (a[0] * g[0] + a[1] * g[1] + a[2] * g[2] + a[3] * g[3]);
        out[1] = s * (a[0] * g[1] + a[1] * g[4] + a[2] * g[5] + a[3] * g[6]);
        out[2] = s * (a[0] * g[2] + a[1] * g[5] + a[2] * g[7] + a[3] * g[8]);
        out[3] = s * (a[0] * g[3] + a[1] * g[6] + a[2] * g[8] + a[3] * g[9]);
    } else {
        const R* g = G.g;
        out[0] = s * (a[0] * g[0] + a[1] * g[1] + a[2] * g[2]);
        out[1] = s * (a[0] * g[1] + a[1] * g[3] + a[2] * g[4]);
        out[2] = s * (a[0] * g[2] + a[1] * g[4] + a[2] * g[5]);
    }
}
// row 0 of G (the product with a = e_0), times s
template <typename R, int D>
__device__ __forceinline__ void grow0(const Gram<R, D>& G, R s, R* out)
{
    if (D == 2) { out[0] = s * G.g[0]; out[1] = s * G.g[1]; out[2] = s * G.g[2]; out[3] = s * G.g[3]; }
    else { out[0] = s * G.g[0]; out[1] = s * G.g[1]; out[2] = s * G.g[2]; }
}

} // namespace cgks
