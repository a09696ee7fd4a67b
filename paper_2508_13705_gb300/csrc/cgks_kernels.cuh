// Stage kernels of the ASE-DFF-CGKS step.  See cgks_device.cuh for the
// mathematics; this file maps it onto grid-stride loops over the work items
// of every mesh in a descriptor table.
//
// Local frame of a direction: dir 0 (faces normal to x): a = i (normal
// index), b = j (tangential); dir 1 (faces normal to y): a = j, b = i.
// Momentum components are ordered normal first in the local frame.
//
// Scratch layouts per mesh and direction (na, nb: cells along / across the
// normal; M Gauss points per face).  Direction 0 as written; direction 1 with
// the two spatial indices swapped, so the global x index is always fastest:
//   FR  [2]{[nb+2][na+1][M][8], [nb+2][na+1][M][4]}
//                                     face states: side 0 = left (from cell f-1),
//                                     side 1 = right (from cell f); per side one
//                                     plane of (W, W_n) pairs, which Step 3 reads
//                                     together, and one plane of W_nn
//   FO  [4][M][nb][na+1][4]           per-point stage outputs (global frame),
//                                     one plane per output quantity and line
//   SP  [nb][na+1][M]                 sigma per face Gauss point (Eq. 3.2)
//   AT  [nb+2][na+6]                  tangential r5 DFF of each cell (Step 3)
//   TD  [nb+2][na+6][8]               FP32 bulk: the cell's tangential differences of hi,
//                                     hi(a, b-1) - hi(a, b) and hi(a, b+1) - hi(a, b), for
//                                     the bases of the Step 3 segments
//
// FP32-bulk form: a cell average W (FP64) is held in the float planes as
// hi = float(W) and lo = float(W - hi), and every reconstructed quantity that
// is a value (line averages, face states, the equilibrium state, the
// interface states) is carried as an increment over the hi of one cell: the
// line average of cell i as lo_i + (its reconstruction's increment), both
// states of a face, its equilibrium state and its interface states as
// increments over hi of the face's right cell.  Stencil
// data enter as differences (hi_k - hi_i) + (lo_k - lo_i), exact in float
// for neighbouring values, so the FP32 arithmetic only ever rounds small
// increments; the O(1) Euler flux of the base hi is formed in float-float in
// the update and the flux of the increment by difference algebra in the
// flux kernel.  The rounding that remains is relative to the increments.
#pragma once
#include "cgks_device.cuh"

namespace cgks {

__device__ __forceinline__ int vglob(int dir, int v) { return dir == 0 ? v : (v == 1 ? 2 : (v == 2 ? 1 : v)); }

template <int M>
__device__ __forceinline__ void local_dims(const Mesh& g, int dir, int& na, int& nb)
{
    na = dir == 0 ? g.nx : g.ny;
    nb = dir == 0 ? g.ny : g.nx;
}

// cell value in local coordinates; lkind: 0 W, 1 W_n (cell), 2 W_t (cell), 3 W_n line,
// 5 the low part of W (FP32-bulk form)
template <int D, int M, typename T, bool WALLS = true>
__device__ __forceinline__ T lcell(const Mesh& g, const T* S, int dir, int lkind, int v, int l, int a, int b,
                                   double tb)
{
    int kind;
    if (lkind == 0 || lkind == 5) kind = lkind;  // W, or its low part (FP32-bulk form)
    else if (lkind == 1) kind = dir == 0 ? 1 : 2;
    else if (lkind == 2) kind = dir == 0 ? 2 : 1;
    else kind = dir == 0 ? 3 : 4;
    int i = dir == 0 ? a : b, j = dir == 0 ? b : a;
    return cell<D, M, T, WALLS>(g, S, kind, vglob(dir, v), l, i, j, tb);
}

// sigma of normal faces (f, b) and of tangential faces of column a (a, f)
template <int D, bool WALLS = true>
__device__ __forceinline__ double lsigN(const Mesh& g, const double* sx, const double* sy, int dir, int f, int b)
{
    return dir == 0 ? sigx<D, WALLS>(g, sx, f, b) : sigy<WALLS>(g, sy, b, f);
}
template <bool WALLS = true>
__device__ __forceinline__ double lsigT(const Mesh& g, const double* sx, const double* sy, int dir, int a, int f)
{
    return dir == 0 ? sigy<WALLS>(g, sy, a, f) : sigx<2, WALLS>(g, sx, f, a);
}

// Scratch indexing.  Direction 0 keeps the normal index a (= i) fastest,
// direction 1 the tangential index b (= i): in both directions the global x
// index runs fastest, in memory and across threads, so every kernel walks the
// SoA state planes with unit stride.
//   cell_idx: a in [-3, na+2], b in [-1, nb]   (AT, TD)
//   fr_row:   bb = b + 1 in [0, nb+1], f in [0, na]   (FR)
//   pt_idx:   b in [0, nb), f in [0, na]       (FO, SP)
__device__ __forceinline__ long long cell_idx(int dir, int na, int nb, int a, int b)
{
    return dir == 0 ? (long long)(b + 1) * (na + 6) + (a + 3) : (long long)(a + 3) * (nb + 2) + (b + 1);
}
__device__ __forceinline__ long long fr_row(int dir, int na, int nb, int bb, int f)
{
    return dir == 0 ? (long long)bb * (na + 1) + f : (long long)f * (nb + 2) + bb;
}
__device__ __forceinline__ long long pt_idx(int dir, int na, int nb, int b, int f)
{
    return dir == 0 ? (long long)b * (na + 1) + f : (long long)f * nb + b;
}
// element offsets of a 16-byte group: FR (point = fr_row * M + l, npt points a
// side) and FO (face = pt_idx, nf faces a plane)
__device__ __forceinline__ long long fr_npt(int na, int nb, int M) { return (long long)(nb + 2) * (na + 1) * M; }
__device__ __forceinline__ long long fr_off(long long npt, long long pt, int side, int nd)
{
    return side * npt * 12 + (nd < 2 ? pt * 8 + nd * 4 : npt * 8 + pt * 4);
}
__device__ __forceinline__ long long fo_off(long long nf, int M, int q, int l, long long face)
{
    return ((long long)(q * M + l) * nf + face) * 4;
}

__device__ __forceinline__ void flag_bad(const Mesh& g, long long idx)
{
    atomicOr(g.status, STATUS_NONPHYS);
    atomicMin((unsigned long long*)g.bad, (unsigned long long)idx);
}

// -------------------------------------------------------------- Steps 1-2 (2-D)
// Step 1 of one cell (a, b) of direction dir: the tangential ASE-DFF
// reconstruction from the five cells b-2..b+2, evaluated at the M Gauss lines
// -> res (line averages; FP32 bulk: lo + the increment over the cell's hi);
// hi: the cell's average (FP32 bulk: its high part).  For the cells whose
// faces this stage evaluates (core), also the tangential r5 DFF (AT, Step 3),
// the tangential differences of hi (TD, FP32 bulk) and the packed DFF of the
// normal stencil (dn, Step 2).
template <int M, typename R, bool WALLS>
__device__ __forceinline__ void step1_cell(const Mesh& g, const R* S, int dir, int na, int nb, int a, int b, double tb,
                                           const double* SX, const double* SY, bool core, R res[M][4], R hi[4],
                                           R dn[4])
{
    constexpr bool BULK32 = sizeof(R) == 4;
    // the tangential stencil: a direct walk for interior cells, whose loads
    // are issued before the DFF selections so that their latencies overlap
    bool inner = a >= 0 && a < na && b >= 2 && b + 2 < nb;
    long long P = g.plane;
    long long ci = dir == 0 ? (long long)b * g.nx + a : (long long)a * g.nx + b;
    long long st = dir == 0 ? g.nx : 1;  // tangential neighbour stride
    int pt = dir == 0 ? 8 : 4;           // plane of the tangential cell slope
    R sw[4][5], swt[4][5], slo[4][BULK32 ? 5 : 1];  // slo: low parts of the averages (FP32 bulk)
    if (inner) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int gv = vglob(dir, v);
            const R* w0 = S + gv * P + ci;
            const R* wt = S + (pt + gv) * P + ci;
            const R* wl = S + (12 + 8 * M + gv) * P + ci;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                sw[v][q] = w0[(q - 2) * st];
                swt[v][q] = wt[(q - 2) * st];
                if (BULK32) slo[v][BULK32 ? q : 0] = wl[(q - 2) * st];
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                sw[v][q] = lcell<2, M, R, WALLS>(g, S, dir, 0, v, 0, a, b + q - 2, tb);
                swt[v][q] = lcell<2, M, R, WALLS>(g, S, dir, 2, v, 0, a, b + q - 2, tb);
                if (BULK32) slo[v][BULK32 ? q : 0] = lcell<2, M, R, WALLS>(g, S, dir, 5, v, 0, a, b + q - 2, tb);
            }
    }
    // face sigma of the tangential stencil: a direct walk for interior cells
    double s6[6];
    if (inner) {
        const double* sp = dir == 0 ? SY + (long long)(b - 2) * g.nx + a : SX + (long long)a * (g.nx + 1) + (b - 2);
        const long long ss = dir == 0 ? g.nx : 1;
#pragma unroll
        for (int q = 0; q < 6; ++q) s6[q] = sp[q * ss];
    } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) s6[q] = lsigT<WALLS>(g, SX, SY, dir, a, b - 2 + q);
    }
    DffR<R> dff = dff_r<R>(dff_select(g.order, s6, g.thr));
    R ht = (R)(dir == 0 ? g.dy : g.dx);
    if (core) {
        long long cidx = cell_idx(dir, na, nb, a, b);
        // tangential r5 DFF of this cell, reused by Step 3 in k_flux
        ((R*)g.AT[dir])[cidx] = (R)dff.a[3];
        if (BULK32) {
            // the tangential differences of hi, for the bases of Step 3's segments
            R tdm[4], tdp[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) { tdm[v] = sw[v][1] - sw[v][2]; tdp[v] = sw[v][3] - sw[v][2]; }
            st4((R*)g.TD[dir] + cidx * 8, tdm);
            st4((R*)g.TD[dir] + cidx * 8 + 4, tdp);
        }
        // the DFF of the normal stencil, used by every Gauss line in Step 2
        double n6[6];
        if (a >= 2 && a + 3 <= na && b >= 0 && b < nb) {
            const double* sp = dir == 0 ? SX + (long long)b * (g.nx + 1) + (a - 2) : SY + (long long)(a - 2) * g.nx + b;
            const long long ss = dir == 0 ? 1 : g.nx;
#pragma unroll
            for (int q = 0; q < 6; ++q) n6[q] = sp[q * ss];
        } else {
#pragma unroll
            for (int q = 0; q < 6; ++q) n6[q] = lsigN<2, WALLS>(g, SX, SY, dir, a - 2 + q, b);
        }
        dff_pack<R>(dff_r<R>(dff_select(g.order, n6, g.thr)), dn);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) hi[v] = sw[v][2];
    const R ghi = (R)g.ghi, glo = (R)g.glo, eps = (R)g.eps;
    with_stencil<M - 2>(dff, [&](auto tag) {
        constexpr int ST = decltype(tag)::value;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            // FP32 bulk: differences of averages as (hi - hi) + (lo - lo), and
            // the line average kept as lo + increment (over the cell's hi)
            R qi = sw[v][2], dp[10];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                dp[q] = BULK32 ? (sw[v][q] - qi) + (slo[v][BULK32 ? q : 0] - slo[v][BULK32 ? 2 : 0]) : sw[v][q] - qi;
                dp[5 + q] = ht * swt[v][q];
            }
            R out[M];
            recon_st<R, M, M - 2, ST, 6>(dff, dp, out, ghi, glo, eps);
            const R base = BULK32 ? slo[v][BULK32 ? 2 : 0] : qi;
#pragma unroll
            for (int l = 0; l < M; ++l) res[l][v] = base + out[l];
        }
    });
}

// Steps 1-2 of one direction, fused through shared memory.  A tile is TA x TB
// cells (a along the face normal, b across it) of the range a in [-1, na],
// b in [-1, nb] whose faces the stage evaluates (ghost columns and rows
// included: Step 3 reads the face states of the rows beside the mesh).  Phase
// 1 runs Step 1 for the tile and two halo columns on each side along a and
// keeps each cell's M line averages, its average and the DFF of its normal
// stencil in shared memory; phase 2 runs Step 2 (Algorithm 1) for every
// (cell, Gauss line) of the tile from there and writes both face states.
// The line averages never reach global memory; the halo costs 4 / TA more
// Step 1 work.  Shared memory per CTA: (TA + 4) TB (4 M + 8) values of R,
// launched as dynamic shared memory.  Shared-memory and thread layouts keep
// the global x index fastest.  Work items are tiles (Work offsets count
// tiles per mesh for the tile shape of the launch).
template <int M, typename R, bool WALLS, int DIR, bool ONE>
__global__ void __launch_bounds__(256) k_recon(Work w, int stage, int TA, int TB)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long cnt[4];
    constexpr bool BULK32 = sizeof(R) == 4;
    constexpr int NV = 4;
    if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
    const int TAH = TA + 4;
    const int ncs = TAH * TB;                       // cells held per tile
    R* s_la = (R*)smem_raw;                         // [M][ncs][4] line averages
    R* s_hi = s_la + (size_t)M * ncs * 4;           // [ncs][4] averages (FP32 bulk: hi)
    R* s_dn = s_hi + (size_t)ncs * 4;               // [ncs][4] packed normal DFF (tile cells)
    const int sa = DIR == 0 ? 1 : TB;               // shared-memory stride of a
    for (long long tile = blockIdx.x; tile < w.total; tile += gridDim.x) {
        long long ltl;
        const Mesh& g = mesh_of<ONE>(w, tile, ltl);
        int na, nb;
        local_dims<M>(g, DIR, na, nb);
        const int nta = (na + 2 + TA - 1) / TA;
        const int lt = (int)ltl;                    // 32-bit tile index (bounded on the host)
        const int a0 = -1 + (lt % nta) * TA, b0 = -1 + (lt / nta) * TB;
        const R* S = state_planes<R>(g, stage == 1 ? 0 : 1);
        const double tb = WALLS ? stage_time(g, stage) : 0.0;  // inflow ghost states
        // sigma of the DFF (Sec. 3.1): of step n-1 in both stages, or, in stage 2
        // of the stage-lag reading, the face means of stage 1 of this step
        const bool lag_stage = stage == 2 && g.dff_lag;
        const double* SX = lag_stage ? g.sig_xn : g.sig_x;
        const double* SY = lag_stage ? g.sig_yn : g.sig_y;
        // ---- phase 1: Step 1 of the tile and its halo along a
        for (int t = threadIdx.x; t < ncs; t += blockDim.x) {
            int ia, ib;
            if (DIR == 0) { ib = t / TAH; ia = t - ib * TAH; }
            else { ia = t / TB; ib = t - ia * TB; }
            const int a = a0 - 2 + ia, b = b0 + ib;
            if (a > na + 2 || b > nb) continue;     // beyond the mesh's halo
            const bool core = ia >= 2 && ia < TA + 2 && a <= na;
            R res[M][4], hi[4], dn[4];
            step1_cell<M, R, WALLS>(g, S, DIR, na, nb, a, b, tb, SX, SY, core, res, hi, dn);
#pragma unroll
            for (int l = 0; l < M; ++l) st4(s_la + ((size_t)l * ncs + t) * 4, res[l]);
            st4(s_hi + (size_t)t * 4, hi);
            if (core) st4(s_dn + (size_t)t * 4, dn);
        }
        __syncthreads();
        // ---- phase 2: Step 2 of every (cell, Gauss line) of the tile
        const R hn = (R)(DIR == 0 ? g.dx : g.dy);
        const R ih = (R)1 / hn;
        const R ghi = (R)g.ghi, glo = (R)g.glo, eps = (R)g.eps;
        R* FR = (R*)g.FR[DIR];
        const long long npt = fr_npt(na, nb, M);
        const long long P = g.plane;
        const int nitem = TA * TB * M;
        for (int it = threadIdx.x; it < nitem; it += blockDim.x) {
            const int l = it % M, c = it / M;
            int ia, ib;
            if (DIR == 0) { ib = c / TA; ia = c - ib * TA + 2; }
            else { ia = c / TB + 2; ib = c - (ia - 2) * TB; }
            const int a = a0 - 2 + ia, b = b0 + ib;
            if (a > na || b > nb) continue;
            const int tc = DIR == 0 ? ib * TAH + ia : ia * TB + ib;
            R pk[4];
            ld4(s_dn + (size_t)tc * 4, pk);
            DffR<R> dff = dff_unpack<R>(pk);
            {
                // branch counts, aggregated per warp
                int bi = dff.st < 0 ? 0 : dff.st - ST_R5 + 1;
                unsigned act = __activemask();
                unsigned same = __match_any_sync(act, bi);
                if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&cnt[bi], (unsigned long long)__popc(same));
            }
            // the line averages and averages of the five stencil cells on this line
            R la5[5][4], sh[5][4];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                ld4(s_la + ((size_t)l * ncs + tc + (q - 2) * sa) * 4, la5[q]);
                ld4(s_hi + (size_t)(tc + (q - 2) * sa) * 4, sh[q]);
            }
            // the normal stencil of line slopes: a direct walk for interior cells
            const bool inner = a >= 2 && a + 2 < na && b >= 0 && b < nb;
            const long long ci = DIR == 0 ? (long long)b * g.nx + a : (long long)a * g.nx + b;
            const long long sn = DIR == 0 ? 1 : g.nx;                  // normal neighbour stride
            const int pl0 = (DIR == 0 ? 12 : 12 + 4 * M) + 4 * l;       // first line-slope plane of line l
            R sl[NV][5];
            if (inner) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const R* ws = S + (pl0 + vglob(DIR, v)) * P + ci;
#pragma unroll
                    for (int q = 0; q < 5; ++q) sl[v][q] = ws[(q - 2) * sn];
                }
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int q = 0; q < 5; ++q) sl[v][q] = lcell<2, M, R, WALLS>(g, S, DIR, 3, v, l, a + q - 2, b, tb);
            }
            R sideL[3][4], sideR[3][4];
            with_stencil<M - 2>(dff, [&](auto tag) {
                constexpr int ST = decltype(tag)::value;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    // FP32 bulk: la5 holds increments over the cells' hi, so a
                    // difference of line averages is (hi - hi) + (la - la), and the
                    // face values come out as increments over this cell's hi
                    R qi = la5[2][v], dp[10];
#pragma unroll
                    for (int q = 0; q < 5; ++q) {
                        dp[q] = BULK32 ? (sh[q][v] - sh[2][v]) + (la5[q][v] - qi) : la5[q][v] - qi;
                        dp[5 + q] = hn * sl[v][q];
                    }
                    R out[6];
                    recon_st<R, 6, M - 2, ST, 0>(dff, dp, out, ghi, glo, eps);
                    // FP32 bulk: the left state of face a+1 over the hi of that face's
                    // right cell a+1, like the right state: a face's two states share a base
                    const R shift = BULK32 ? sh[2][v] - sh[3][v] : (R)0;
                    sideL[0][v] = (qi + shift) + out[0]; sideL[1][v] = out[1] * ih; sideL[2][v] = out[2] * ih * ih;
                    sideR[0][v] = qi + out[3]; sideR[1][v] = out[4] * ih; sideR[2][v] = out[5] * ih * ih;
                }
            });
            // side 0: left state of face a+1 (value at xi = +1/2)
            if (a + 1 <= na) {
                long long pt = fr_row(DIR, na, nb, b + 1, a + 1) * M + l;
#pragma unroll
                for (int nd = 0; nd < 3; ++nd) st4(FR + fr_off(npt, pt, 0, nd), sideL[nd]);
            }
            // side 1: right state of face a (value at xi = -1/2)
            if (a >= 0) {
                long long pt = fr_row(DIR, na, nb, b + 1, a) * M + l;
#pragma unroll
                for (int nd = 0; nd < 3; ++nd) st4(FR + fr_off(npt, pt, 1, nd), sideR[nd]);
            }
        }
        __syncthreads();  // the next tile reuses the shared memory
    }
    if (threadIdx.x < 4 && cnt[threadIdx.x] && w.n > 0)
        atomicAdd(&(ONE ? w.m0 : w.mesh[0]).branch[threadIdx.x], cnt[threadIdx.x]);
}

// -------------------------------------------------------------- Step 2 (1-D)
// The reconstruction of a 1-D cell a in [-1, nx] from the cell averages and
// slopes of a-2..a+2: the right state of face a and the left state of face a+1.
template <typename R, bool WALLS, bool ONE>
__global__ void __launch_bounds__(256) k_normal1(Work w, int stage)
{
    __shared__ unsigned long long cnt[4];
    if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
    __syncthreads();
    constexpr int NV = 3;
    constexpr bool BULK32 = sizeof(R) == 4;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        long long li;
        const Mesh& g = mesh_of<ONE>(w, gi, li);
        const int a = (int)li - 1;
        const int na = g.nx;
        const R* S = state_planes<R>(g, stage == 1 ? 0 : 1);
        const double tb = WALLS ? stage_time(g, stage) : 0.0;  // inflow ghost states
        double s6[6];
        // sigma of the DFF: step n-1, or in stage 2 of the stage-lag reading the
        // face means of stage 1 of this step
        const double* SX = (stage == 2 && g.dff_lag) ? g.sig_xn : g.sig_x;
#pragma unroll
        for (int q = 0; q < 6; ++q) s6[q] = sigx<1, WALLS>(g, SX, a - 2 + q, 0);
        DffR<R> dff = dff_r<R>(dff_select(g.order, s6, g.thr));
        {
            // branch counts, aggregated per warp
            int bi = dff.st < 0 ? 0 : dff.st - ST_R5 + 1;
            unsigned act = __activemask();
            unsigned same = __match_any_sync(act, bi);
            if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&cnt[bi], (unsigned long long)__popc(same));
        }
        const R hn = (R)g.dx;
        const R ih = (R)1 / hn;
        const R ghi = (R)g.ghi, glo = (R)g.glo, eps = (R)g.eps;
        R sideL[3][4], sideR[3][4];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            // FP32 bulk: differences as (hi - hi) + (lo - lo); the face values
            // come out as increments over this cell's hi (qi = lo)
            R qi = cell<1, 1, R, WALLS>(g, S, 0, v, 0, a, 0, tb);
            R ql = BULK32 ? cell<1, 1, R, WALLS>(g, S, 5, v, 0, a, 0, tb) : (R)0;
            R dp[10];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                dp[q] = cell<1, 1, R, WALLS>(g, S, 0, v, 0, a + q - 2, 0, tb) - qi;
                if (BULK32) dp[q] += cell<1, 1, R, WALLS>(g, S, 5, v, 0, a + q - 2, 0, tb) - ql;
                dp[5 + q] = hn * cell<1, 1, R, WALLS>(g, S, 1, v, 0, a + q - 2, 0, tb);
            }
            // the left state of face a+1 over hi of cell a+1 (a face's states share a base)
            const R shift = BULK32 ? qi - cell<1, 1, R, WALLS>(g, S, 0, v, 0, a + 1, 0, tb) : (R)0;
            if (BULK32) qi = ql;
            R out[6];
            recon<R, 6>(dff, g.oi, 0, dp, out, ghi, glo, eps);
            sideL[0][v] = (qi + shift) + out[0]; sideL[1][v] = out[1] * ih; sideL[2][v] = out[2] * ih * ih;
            sideR[0][v] = qi + out[3]; sideR[1][v] = out[4] * ih; sideR[2][v] = out[5] * ih * ih;
        }
#pragma unroll
        for (int nd = 0; nd < 3; ++nd) { sideL[nd][3] = (R)0; sideR[nd][3] = (R)0; }
        R* FR = (R*)g.FR[0];
        const long long npt = fr_npt(na, 1, 1);
        // side 0: left state of face a+1 (value at xi = +1/2)
        if (a + 1 <= na) {
            long long pt = fr_row(0, na, 1, 1, a + 1);
#pragma unroll
            for (int nd = 0; nd < 3; ++nd) st4(FR + fr_off(npt, pt, 0, nd), sideL[nd]);
        }
        // side 1: right state of face a (value at xi = -1/2)
        if (a >= 0) {
            long long pt = fr_row(0, na, 1, 1, a);
#pragma unroll
            for (int nd = 0; nd < 3; ++nd) st4(FR + fr_off(npt, pt, 1, nd), sideR[nd]);
        }
    }
    __syncthreads();
    if (threadIdx.x < 4 && cnt[threadIdx.x] && w.n > 0)
        atomicAdd(&(ONE ? w.m0 : w.mesh[0]).branch[threadIdx.x], cnt[threadIdx.x]);
}

// -------------------------------------------------------------- Step 3 + flux
// One thread per face Gauss point.  The two sides stream through one at a
// time: each side's reconstructed data (Step 2 values, Step 3 tangential
// derivatives), its Maxwellian half-range moments and micro-slopes are folded
// into the kinetic weighting Q0, dQ0 (Eq. 2.7) and the half-range terms of
// Eq. 2.6 as soon as they are formed, so only one side is live at a time.
// CAP = 1 asks for at least 4 resident blocks of 128 threads (<= 128 registers,
// spilling the rest); CAP = 0 for 3 in FP32 (<= 170 registers) and 1 in FP64.
// The autotuner times both variants in FP64, where they round alike; the
// FP32-bulk form has the uncapped one only (a capped compilation may contract
// its FP32 arithmetic differently, and results must not depend on tuning).  HG = 1 compiles the
// collision-time terms (tau > 0); the tau = 0 instance leaves them out and
// carries fewer live values.  PF = true compiles the first-order fallback at
// face points whose reconstructed state is not physical (a flagged option).
template <int D, int M, typename R, int STAGE, int CAP, int HG, bool PF, bool ONE>
__global__ void __launch_bounds__(128, CAP ? 4 : (sizeof(R) == 4 ? (HG ? 3 : 4) : 1)) k_flux(Work w)
{
    constexpr int NV = D + 2;
    constexpr int ND = D == 2 ? 5 : 2;  // derivatives: n, nn (, t, tt, nt)
    constexpr bool BULK32 = sizeof(R) == 4;
    // FP32 bulk: the two sides unrolled, so that their independent chains
    // interleave, and Step 3's segment loop rolled, which keeps the tau = 0
    // compilation within 128 registers without spills (4 blocks of 128
    // threads per SM; the tau > 0 ones take 168, 3 blocks)
    constexpr int kSides = BULK32 ? 2 : 1, kSegs = BULK32 ? 1 : 3;
    // Step 3 weights in shared memory: the Gauss line differs across the lanes
    // of a warp, which would serialise constant-memory reads.  FP32 bulk also
    // keeps, per line and segment, the sum of the segment's weights, which
    // multiplies the difference of the segment cell's hi from the centre's.
    __shared__ R s_d1[4][12], s_d2[4][12];
    __shared__ R s_c1[4][3], s_c2[4][3];
    if (D == 2) {
        const auto& T = Tab<R>::get((ONE ? w.m0 : w.mesh[0]).oi);  // a table shares one order
        for (int q = threadIdx.x; q < 48; q += blockDim.x) {
            s_d1[q / 12][q % 12] = T.d1[q / 12][q % 12];
            s_d2[q / 12][q % 12] = T.d2[q / 12][q % 12];
        }
        if (BULK32)
            for (int q = threadIdx.x; q < 12; q += blockDim.x) {
                R c1 = 0, c2 = 0;
                for (int kk = 0; kk < M; ++kk) { c1 += T.d1[q / 3][(q % 3) * M + kk]; c2 += T.d2[q / 3][(q % 3) * M + kk]; }
                s_c1[q / 3][q % 3] = c1;
                s_c2[q / 3][q % 3] = c2;
            }
        __syncthreads();
    }
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        long long lil;
        const Mesh& g = mesh_of<ONE>(w, gi, lil);
        unsigned li = (unsigned)lil;  // 32-bit local index (bounded on the host)
        int dir = 0, na = g.nx, nb = 1;
        if (D == 2) {
            unsigned nxl = (unsigned)(g.nx + 1) * (unsigned)g.ny * M;
            dir = li < nxl ? 0 : 1;
            if (dir == 1) li -= nxl;
            local_dims<M>(g, dir, na, nb);
        }
        int l = D == 2 ? (int)(li % M) : 0;
        unsigned r = D == 2 ? li / M : li;
        int f, b;
        if (D == 1) { f = (int)r; b = 0; }
        else if (dir == 0) { unsigned d = na + 1, q = r / d; f = (int)(r - q * d); b = (int)q; }
        else { unsigned d = nb, q = r / d; b = (int)(r - q * d); f = (int)q; }
        const R* FR = (const R*)g.FR[dir];
        const R gm = MeshR<R>::gamma(g), K = MeshR<R>::K(g);
        constexpr bool hgks = HG != 0;  // the collision-time terms of Eq. 2.6 (tau > 0)
        const long long npt = fr_npt(na, nb, M);
        const long long p00 = fr_row(dir, na, nb, b, f) * M;
        const long long rs = (dir == 0 ? (long long)(na + 1) : 1LL) * M;  // FR row stride of the segments
        // FP32 bulk: the state planes of this stage, whose high part hi of the
        // face's right cell f is the base of both face states (local frame)
        const R* SF = state_planes<R>(g, STAGE == 1 ? 0 : 1);
        const double tb = stage_time(g, STAGE);
        // hb1: hi of the right cell f, the base of both face states
        R hb1[4] = {0, 0, 0, 0};
        if (BULK32) {
            if (f < na && (D == 1 || b < nb)) {
                long long ci = dir == 0 ? (long long)b * g.nx + f : (long long)f * g.nx + b;
#pragma unroll
                for (int v = 0; v < NV; ++v) hb1[v] = SF[vglob(dir, v) * g.plane + ci];
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) hb1[v] = lcell<D, M, R, true>(g, SF, dir, 0, v, 0, f, b, tb);
            }
        }
        // FP32 bulk: whether the jump W_l - W_r is small enough for the kinetic
        // weighting to be taken to first order in it (decided with the left
        // state, below); the first-order term, held in Q0 itself unless the
        // point fallback may still change the states
        bool lin = false;
        R Dl[4] = {0, 0, 0, 0};
        R e1v[4] = {1, 0, 0, 0};
        R Q0[4] = {0, 0, 0, 0};
        R dQ[ND][4];
#pragma unroll
        for (int q = 0; q < ND; ++q)
#pragma unroll
            for (int v = 0; v < 4; ++v) dQ[q][v] = 0;
        R T5[4] = {0, 0, 0, 0}, T6[4] = {0, 0, 0, 0}, S1h[4] = {0, 0, 0, 0};
        R pz[2], mn[2], mt[2];
        bool bad = false, ok = true;
#pragma unroll kSides
        for (int side = 0; side < 2; ++side) {
            // Step 2 data: W, W_n, W_nn (FP32 bulk: W as an increment over hb1);
            // Step 3's tangential derivatives are formed later, right before
            // their micro-slope solves, so that few derivatives are live at once
            R d0[4], dn[2][4];
            const int a = side == 0 ? f - 1 : f;  // the reconstructing cell
            const R* Fs = FR + side * npt * 12 + p00 * 8;  // (W, W_n) of segment b - 1
            ld4(Fs + (rs + l) * 8, d0);
            ld4(Fs + (rs + l) * 8 + 4, dn[0]);
            ld4(FR + side * npt * 12 + npt * 8 + (p00 + rs + l) * 4, dn[1]);
            // the side's state
            R ws[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) ws[v] = BULK32 ? hb1[v] + d0[v] : d0[v];
            bool fb = false;  // the side fell back to its cell average (all derivatives zero)
            if (PF) {
                // fallback: a side whose point state has rho <= 0 or p <= 0 takes
                // the average of the cell it was reconstructed from, first order;
                // the test is made in FP64 (FP32 bulk: on hi + increment)
                double W4[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) W4[v] = BULK32 ? (double)hb1[v] + (double)d0[v] : (double)d0[v];
                double rho = W4[0];
                double m2 = W4[1] * W4[1] + (D == 2 ? W4[2] * W4[2] : 0.0);
                double p = (g.gamma - 1.0) * (W4[NV - 1] - 0.5 * m2 / rho);
                if (!(rho > 0.0) || !(p > 0.0)) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        // FP32 bulk: the average over hb1, (hi_a - hb1) + lo_a
                        if (BULK32)
                            d0[v] = (side == 0 ? lcell<D, M, R, true>(g, SF, dir, 0, v, 0, a, b, tb) - hb1[v] : (R)0)
                                  + lcell<D, M, R, true>(g, SF, dir, 5, v, 0, a, b, tb);
                        else
                            d0[v] = lcell<D, M, R, true>(g, SF, dir, 0, v, 0, a, b, tb);
                        ws[v] = BULK32 ? hb1[v] + d0[v] : d0[v];
                        dn[0][v] = dn[1][v] = (R)0;
                    }
                    fb = true;
                    lin = false;  // the states changed: weight them directly
                    atomicAdd(g.nfall, 1ull);
                }
            }
            // Eq. 3.2 ingredients and the positivity test, in the precision the
            // states carry (the face means, stencil sums and branch thresholds
            // that use sigma are FP64)
            {
                R rho = ws[0];
                R ir = (R)1 / rho;
                R un = ws[1] * ir;
                R ut = D == 2 ? ws[2] * ir : (R)0;
                R p = (gm - (R)1) * (ws[NV - 1] - (R)0.5 * rho * (un * un + ut * ut));
                R ic = (R)1 / sqrt(gm * p * ir);
                pz[side] = p; mn[side] = un * ic; mt[side] = ut * ic;
                bad |= !(rho > (R)0) || !(p > (R)0);
            }
            // kinetic weighting (Eq. 2.7): this side's half-range integrals
            Mom<R, D> Ms;
            ok &= maxwellian<R, D>(ws, gm, K, side == 0 ? 1 : 2, Ms);
            Gram<R, D> Gs;  // half-range <psi psi> of this side
            gram<R, D, 0, 0>(Ms, Gs);
            R t[4], z[4];
            grow0<R, D>(Gs, Ms.rho, t);
            if (BULK32 && side == 0) {
                // Q0 = W_r + (H(W_l) - H(W_r)), H the u > 0 half-range moments;
                // for a small jump, H(W_l) - H(W_r) = dH/dW (W_l - W_r) to second
                // order, where dH/dW dW = <psi a>_{u > 0} with <a> = dW: the
                // rounding then stays relative to the jump.  W_l - W_r is the
                // difference of the two increments (a face's states share a base).
                R e1[4], dW[4];
                ld4(FR + npt * 12 + (p00 + rs + l) * 8, e1);
                const R sc = fabs(hb1[0]) + fabs(hb1[NV - 1]);
                lin = true;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    dW[v] = d0[v] - e1[v];
                    lin &= fabs(dW[v]) <= (R)2.5e-4 * sc;
                }
                if (NV < 4) dW[3] = (R)0;
                if (lin) {
                    R aa[4];
                    slope<R, D>(Ms, K, dW, aa);
                    gmul<R, D>(Gs, aa, Ms.rho, PF ? Dl : Q0);
                }
            }
            if (!(BULK32 && lin && !PF)) {
#pragma unroll
                for (int v = 0; v < NV; ++v) Q0[v] += t[v];
            }
            if (hgks) {
                mom<R, D>(Ms, e1v, 1, 0, t);
#pragma unroll
                for (int v = 0; v < NV; ++v) T5[v] += Ms.rho * t[v];
            }
            // one derivative: its micro-slope (<a> = dW of this side, Eq. 2.8)
            // into the weighted derivative dQ[q], and for q = 0 (n) and 2 (t) the
            // half-range (a_n u + a_t v) terms of Eq. 2.6 with and without the
            // flux's u
            auto fold = [&](int q, const R dv[4]) {
                R a_[4];
                slope<R, D>(Ms, K, dv, a_);
                gmul<R, D>(Gs, a_, Ms.rho, t);
#pragma unroll
                for (int v = 0; v < NV; ++v) dQ[q][v] += t[v];
                if (hgks && (q == 0 || (D == 2 && q == 2))) {
                    int pu = q == 0 ? 1 : 0, pv = q == 0 ? 0 : 1;
                    mom<R, D>(Ms, a_, pu, pv, t);
                    mom<R, D>(Ms, a_, pu + 1, pv, z);
#pragma unroll
                    for (int v = 0; v < NV; ++v) { S1h[v] += Ms.rho * t[v]; T6[v] += Ms.rho * z[v]; }
                }
            };
            fold(0, dn[0]);
            fold(1, dn[1]);
            if (D == 2) {
                // Step 3: tangential derivatives from the 3M face points of
                // segments b-1, b, b+1, scaled by the tangential r5 DFF of the
                // reconstructing cell (a = f-1 for the left state, f for the right)
                R at = ((const R*)g.AT[dir])[cell_idx(dir, na, nb, a, b)];
                R iht = (R)1 / (R)(dir == 0 ? g.dy : g.dx);
                R c1 = fb ? (R)0 : at * iht, c2 = fb ? (R)0 : at * iht * iht;
                {
                    // W_t and W_tt from the points' values
                    R wt[4] = {0, 0, 0, 0}, wtt[4] = {0, 0, 0, 0};
#pragma unroll kSegs
                    for (int s = 0; s < 3; ++s)
#pragma unroll
                        for (int kk = 0; kk < M; ++kk) {
                            R x0[4];
                            ld4(Fs + (s * rs + kk) * 8, x0);
                            R w1 = s_d1[l][s * M + kk], w2 = s_d2[l][s * M + kk];
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                wt[v] += w1 * x0[v];
                                wtt[v] += w2 * x0[v];
                            }
                        }
                    if (BULK32) {
                        // the segment points' values are increments over hi of the
                        // right cells (f, b-1), (f, b), (f, b+1): add the bases' part
                        // from their differences (the weights of a constant sum to zero)
                        R dm[4], dpl[4];
                        const R* td = (const R*)g.TD[dir] + cell_idx(dir, na, nb, f, b) * 8;
                        ld4(td, dm);
                        ld4(td + 4, dpl);
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            wt[v] += s_c1[l][0] * dm[v] + s_c1[l][2] * dpl[v];
                            wtt[v] += s_c2[l][0] * dm[v] + s_c2[l][2] * dpl[v];
                        }
                    }
#pragma unroll
                    for (int v = 0; v < 4; ++v) { wt[v] *= c1; wtt[v] *= c2; }
                    fold(2, wt);
                    fold(3, wtt);
                }
                {
                    // W_nt from the points' normal derivatives
                    R wnt[4] = {0, 0, 0, 0};
#pragma unroll kSegs
                    for (int s = 0; s < 3; ++s)
#pragma unroll
                        for (int kk = 0; kk < M; ++kk) {
                            R x1[4];
                            ld4(Fs + (s * rs + kk) * 8 + 4, x1);
                            R w1 = s_d1[l][s * M + kk];
#pragma unroll
                            for (int v = 0; v < 4; ++v) wnt[v] += w1 * x1[v];
                        }
#pragma unroll
                    for (int v = 0; v < 4; ++v) wnt[v] *= c1;
                    fold(4, wnt);
                }
            }
        }
        // FP32 bulk: the equilibrium state as an increment qv over hb1
        R qv[4] = {0, 0, 0, 0};
        if (BULK32) {
            if (lin) {
                R e1[4];
                ld4(FR + npt * 12 + (p00 + rs + l) * 8, e1);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    qv[v] = e1[v] + (PF ? Dl[v] : Q0[v]);
                    Q0[v] = hb1[v] + qv[v];
                }
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) qv[v] = Q0[v] - hb1[v];
            }
        }
        double sig;
        {
            R dpz = fabs(pz[0] - pz[1]);
            sig = (double)(dpz / pz[0] + dpz / pz[1] + (mn[0] - mn[1]) * (mn[0] - mn[1]) + (mt[0] - mt[1]) * (mt[0] - mt[1]));
        }
        // equilibrium state g0 and its micro-slopes, time derivatives (Eq. 2.8)
        const R Dt = MeshR<R>::dt(g);
        Mom<R, D> M0;
        ok &= maxwellian<R, D>(Q0, gm, K, 0, M0);
        // <u psi psi> and <v psi psi> of g0 serve every u- and v-weighted moment below
        Gram<R, D> Gu, Gv;
        gram<R, D, 1, 0>(M0, Gu);
        if (D == 2) gram<R, D, 0, 1>(M0, Gv);
        R S1[4], S2[4], z[4], rhs[4], Ab[4], A1t[4], A2t[4] = {0, 0, 0, 0};
        R an[4], at2[4];
        slope<R, D>(M0, K, dQ[0], an);
        gmul<R, D>(Gu, an, (R)1, S1);
        if (D == 2) {
            slope<R, D>(M0, K, dQ[2], at2);
            gmul<R, D>(Gv, at2, (R)1, z);
#pragma unroll
            for (int v = 0; v < NV; ++v) S1[v] += z[v];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) { S1[v] *= M0.rho; rhs[v] = -S1[v]; }
        slope<R, D>(M0, K, rhs, Ab);
        {
            R ann[4];
            slope<R, D>(M0, K, dQ[1], ann);
            gmul<R, D>(Gu, ann, (R)1, rhs);
        }
        if (D == 2) {
            R ant[4];
            slope<R, D>(M0, K, dQ[4], ant);
            gmul<R, D>(Gv, ant, (R)1, z);
#pragma unroll
            for (int v = 0; v < NV; ++v) rhs[v] += z[v];
            R s2[4];
            gmul<R, D>(Gu, ant, (R)1, s2);
#pragma unroll
            for (int v = 0; v < NV; ++v) rhs[v] *= -M0.rho;
            slope<R, D>(M0, K, rhs, A1t);
            R att[4];
            slope<R, D>(M0, K, dQ[3], att);
            gmul<R, D>(Gv, att, (R)1, z);
#pragma unroll
            for (int v = 0; v < NV; ++v) rhs[v] = -M0.rho * (s2[v] + z[v]);
            slope<R, D>(M0, K, rhs, A2t);
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) rhs[v] *= -M0.rho;
            slope<R, D>(M0, K, rhs, A1t);
        }
        gmul<R, D>(Gu, A1t, (R)1, S2);
        if (D == 2) {
            gmul<R, D>(Gv, A2t, (R)1, z);
#pragma unroll
            for (int v = 0; v < NV; ++v) S2[v] += z[v];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) S2[v] *= M0.rho;
        // flux terms <u> and <A u>; the linear / quadratic fits of Eq. 2.19-2.20
        // and 2.29 reduce to F = <u>, F_t = <A u>, W_t = -S1, W_tt = -S2 at tau = 0
        R F[4], Ft[4], Wt[4], Wtt[4];
        grow0<R, D>(Gu, (R)1, F);
        gmul<R, D>(Gu, Ab, (R)1, Ft);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            F[v] *= M0.rho;
            Ft[v] *= M0.rho;
            Wt[v] = -S1[v];
            Wtt[v] = -S2[v];
        }
        // the flux carried out: F itself (FP64), or its increment over the Euler
        // flux of hb1 (FP32 bulk; that flux is added in the update): the Euler
        // flux of Q0 = hb1 + qv taken as a difference
        R Fo[4];
        if (BULK32) euler_flux_delta<D>(hb1, qv, gm - (R)1, Fo);
        else {
#pragma unroll
            for (int v = 0; v < 4; ++v) Fo[v] = F[v];
        }
        if (hgks) {
            // inviscid: c1 dt; viscous (Sec. 4): mu / p with p the pressure of
            // the equilibrium state at the face point
            R base = g.tau_mode == 2 ? MeshR<R>::mu(g) / (M0.rho * M0.il) : MeshR<R>::c1(g) * Dt;
            R tau = base + MeshR<R>::c2(g) * fabs(pz[0] - pz[1]) / (pz[0] + pz[1]) * Dt;
            // collision and non-equilibrium terms of Eq. 2.6, fitted analytically
            R Att[4], T2[4], T3[4], T4[4];
#pragma unroll
            for (int v = 0; v < NV; ++v) rhs[v] = -S2[v];
            slope<R, D>(M0, K, rhs, Att);
            gmul<R, D>(Gu, Att, (R)1, T2);
            mom<R, D>(M0, an, 2, 0, T3);
            mom<R, D>(M0, A1t, 2, 0, T4);
            if (D == 2) {
                mom<R, D>(M0, at2, 1, 1, z);
#pragma unroll
                for (int v = 0; v < NV; ++v) T3[v] += z[v];
                mom<R, D>(M0, A2t, 1, 1, z);
#pragma unroll
                for (int v = 0; v < NV; ++v) T4[v] += z[v];
            }
            R ed = exp(-Dt / tau), eh = exp((R)-0.5 * Dt / tau);
            R h = (R)0.5 * Dt;
            R E0d = tau * ((R)1 - ed), E0h = tau * ((R)1 - eh);
            R E1d = tau * tau * ((R)1 - ed) - tau * Dt * ed, E1h = tau * tau * ((R)1 - eh) - tau * h * eh;
            R f0 = ((R)4 * E0h - E0d) / Dt, g0 = (R)4 * (E0d - (R)2 * E0h) / (Dt * Dt);
            R f1 = ((R)4 * E1h - E1d) / Dt, g1 = (R)4 * (E1d - (R)2 * E1h) / (Dt * Dt);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                R T3s = T3[v] * M0.rho, T4s = T4[v] * M0.rho, T2s = T2[v] * M0.rho;
                R T0v = F[v], T1v = Ft[v];
                // F = T0 + (the terms below); FP32 bulk adds them to the increment
                Fo[v] += -f0 * T0v - tau * T1v + (f1 - tau) * T3s + f0 * T5[v] - f1 * T6[v];
                Ft[v] = -g0 * T0v + T1v - tau * T2s + g1 * T3s - tau * T4s + g0 * T5[v] - g1 * T6[v];
                R dS = S1[v] - S1h[v];
                Wt[v] += ((R)2 * eh - ed) * dS;
                Wtt[v] += (R)4 * (ed - eh) / Dt * dS;
            }
        }
        long long face = pt_idx(dir, na, nb, b, f);
        long long pt = face * M + l;  // SP index
        const long long nf = (long long)nb * (na + 1);
        R* FO = (R*)g.FO[dir];
        R o[4][4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int gv = D == 2 ? vglob(dir, v) : v;
            if (v >= NV) { o[0][v] = o[1][v] = o[2][v] = o[3][v] = (R)0; continue; }
            // interface-state values: Q0 itself, or its increment over hb1 (FP32 bulk)
            const R Qv = BULK32 ? qv[v] : Q0[v];
            if (STAGE == 1) {
                o[0][gv] = (R)0.5 * Dt * Fo[v] + (R)0.125 * Dt * Dt * Ft[v];
                o[1][gv] = Dt * Fo[v] + Dt * Dt / (R)6 * Ft[v];
                o[2][gv] = Qv + (R)0.5 * Dt * Wt[v] + (R)0.125 * Dt * Dt * Wtt[v];
                o[3][gv] = Qv + Dt * Wt[v] + Dt * Dt / (R)6 * Wtt[v];
            } else {
                o[0][gv] = Dt * Dt / (R)3 * Ft[v];
                o[1][gv] = Dt * Dt / (R)3 * Wtt[v];
            }
        }
        bool finite = true;
        constexpr int NO = STAGE == 1 ? 4 : 2;
#pragma unroll
        for (int q = 0; q < NO; ++q) {
#pragma unroll
            for (int v = 0; v < NV; ++v) finite &= isfinite(o[q][v]);
            st4(FO + fo_off(nf, M, q, l, face), o[q]);
        }
        if (STAGE == 1) g.SP[dir][pt] = sig;
        if (bad || !ok || !finite) flag_bad(g, pt);
    }
}

// -------------------------------------------------------------- update (2-D)
// r - l exactly, as a double: in FP64 the difference itself; in FP32 the
// rounded difference plus its rounding error (Knuth's two-sum), each exact
// in a double.
__device__ __forceinline__ double exact_diff(double r, double l) { return r - l; }
__device__ __forceinline__ double exact_diff(float r, float l)
{
    float b = -l;
    float s = r + b;
    float z = s - r;
    float e = (r - (s - z)) + (b - z);
    return (double)s + (double)e;
}

// Stage 1 writes W* (S1) and the accumulator; stage 2 writes state n+1 (S0).
// FP32-bulk form: the float planes (F1 / F0) receive everything the next stage
// reads, the FP64 planes the cell averages of state n+1 (W* lives in F1 only).
template <int M, typename R, int STAGE, bool ONE>
__global__ void __launch_bounds__(256) k_update2(Work w)
{
    constexpr bool BULK32 = sizeof(R) == 4;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        long long c;
        const Mesh& g = mesh_of<ONE>(w, gi, c);
        unsigned cu = (unsigned)c, qj = cu / (unsigned)g.nx;  // 32-bit (bounded on the host)
        int i = (int)(cu - qj * (unsigned)g.nx), j = (int)qj;
        const R* FX = (const R*)g.FO[0];
        const R* FY = (const R*)g.FO[1];
        // x-faces: b = j, f = i and i+1; y-faces: b = i, f = j and j+1
        const long long fxl = (long long)j * (g.nx + 1) + i, fyl = (long long)j * g.nx + i;
        const long long nfx = (long long)g.ny * (g.nx + 1), nfy = (long long)g.nx * (g.ny + 1);
        const double idx = g.idx, idy = g.idy;
        const R ridx = MeshR<R>::ih(g, 0), ridy = MeshR<R>::ih(g, 1);
        long long P = g.plane;
        double* out = STAGE == 1 ? g.S1 : g.S0;
        // line-slope part of the accumulator, held in the bulk precision (a float
        // view in the FP32-bulk form: it only ever holds bulk values)
        R* accs = (R*)(g.ACC + 4 * P);
        float* outf = STAGE == 1 ? g.F1 : g.F0;
        const auto& TR = Tab<R>::get(g.oi);
        // Conserved quantities: the Gauss sum over a face's points is formed
        // per face, in the bulk precision and in the same order by both cells
        // of the face (bitwise alike), and the difference of a cell's two
        // face sums is taken exactly (exact_diff) into the FP64 averages, so
        // the updates telescope over the mesh and the totals change only by
        // the boundary fluxes and FP64 rounding.  Slopes use bulk differences.
        // FP32 bulk, stage 1: the face outputs are increments over hi of each
        // face's right cell (this cell for the left and bottom faces, cells
        // (i+1, j) and (i, j+1) for the others).  Their flux parts add
        // dt/2 (F(hi_R) - F(hi_L)) and dt (...) with the Euler fluxes F of the
        // bases in float-float (each cell forms the same values bitwise, so
        // the update still telescopes), their state parts the difference of
        // the bases' hi.
        R h0[4] = {0, 0, 0, 0}, hxn[4] = {0, 0, 0, 0}, hyn[4] = {0, 0, 0, 0};
        ff Bx[4], By[4];
        if (BULK32 && STAGE == 1) {
            const float* SF = g.F0;
            const double tb = *g.tn;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                h0[v] = (R)SF[v * P + c];
                hxn[v] = (R)cell<2, M, float, true>(g, SF, 0, v, 0, i + 1, j, tb);
                hyn[v] = (R)cell<2, M, float, true>(g, SF, 0, v, 0, i, j + 1, tb);
            }
            const double gm1d = g.gamma - 1.0;
            const ff gm1 = {(float)gm1d, (float)(gm1d - (double)(float)gm1d)};
            ff f0[4], f1[4];
            float wl[4];
            // x: local frame = global (rho, m_x, m_y, E)
            for (int v = 0; v < 4; ++v) wl[v] = (float)h0[v];
            euler_flux_ff<2>(wl, gm1, f0);
            for (int v = 0; v < 4; ++v) wl[v] = (float)hxn[v];
            euler_flux_ff<2>(wl, gm1, f1);
            for (int v = 0; v < 4; ++v) Bx[v] = ff_add(f1[v], ff_neg(f0[v]));
            // y: local frame (rho, m_y, m_x, E), back to global order
            wl[0] = (float)h0[0]; wl[1] = (float)h0[2]; wl[2] = (float)h0[1]; wl[3] = (float)h0[3];
            euler_flux_ff<2>(wl, gm1, f0);
            wl[0] = (float)hyn[0]; wl[1] = (float)hyn[2]; wl[2] = (float)hyn[1]; wl[3] = (float)hyn[3];
            euler_flux_ff<2>(wl, gm1, f1);
            const int yl[4] = {0, 2, 1, 3};
            for (int v = 0; v < 4; ++v) By[v] = ff_add(f1[yl[v]], ff_neg(f0[yl[v]]));
        }
        R gxr0[4] = {0, 0, 0, 0}, gxl0[4] = {0, 0, 0, 0}, gyr0[4] = {0, 0, 0, 0}, gyl0[4] = {0, 0, 0, 0};
        R gxr1[4] = {0, 0, 0, 0}, gxl1[4] = {0, 0, 0, 0}, gyr1[4] = {0, 0, 0, 0}, gyl1[4] = {0, 0, 0, 0};
        R sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
#pragma unroll 1
        for (int l = 0; l < M; ++l) {
            R wl = TR.gw[l];
            R a[4], bq[4], cq[4], dq[4];
            // stage 1: o0 = F(dt/2), o1 = dt F + dt^2/6 F_t, o2 = W(dt/2), o3 = W0 + dt W_t + dt^2/6 W_tt
            // stage 2: o0 = dt^2/3 F_t*, o1 = dt^2/3 W_tt*
#pragma unroll
            for (int q = 0; q < (STAGE == 1 ? 4 : 2); ++q) {
                ld4(FX + fo_off(nfx, M, q, l, fxl + 1), a);
                ld4(FX + fo_off(nfx, M, q, l, fxl), bq);
                ld4(FY + fo_off(nfy, M, q, l, fyl + g.nx), cq);
                ld4(FY + fo_off(nfy, M, q, l, fyl), dq);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    R dx_ = a[v] - bq[v];
                    R dy_ = cq[v] - dq[v];
                    if (BULK32 && STAGE == 1 && q >= 2) {  // interface states over the bases' hi
                        dx_ += hxn[v] - h0[v];
                        dy_ += hyn[v] - h0[v];
                    }
                    if (q == 0) {
                        gxr0[v] += wl * a[v]; gxl0[v] += wl * bq[v];
                        gyr0[v] += wl * cq[v]; gyl0[v] += wl * dq[v];
                    } else if (STAGE == 1 && q == 1) {
                        gxr1[v] += wl * a[v]; gxl1[v] += wl * bq[v];
                        gyr1[v] += wl * cq[v]; gyl1[v] += wl * dq[v];
                    } else if ((STAGE == 1 && q == 2) || (STAGE == 2 && q == 1)) {
                        R lx = dx_ * ridx, ly = dy_ * ridy;
                        if (STAGE == 2) {
                            lx += accs[(4 * l + v) * P + c];
                            ly += accs[(4 * M + 4 * l + v) * P + c];
                        }
                        if (BULK32) {
                            outf[(12 + 4 * l + v) * P + c] = (float)lx;
                            outf[(12 + 4 * M + 4 * l + v) * P + c] = (float)ly;
                        } else {
                            out[(12 + 4 * l + v) * P + c] = (double)lx;
                            out[(12 + 4 * M + 4 * l + v) * P + c] = (double)ly;
                        }
                        sx[v] += wl * lx;
                        sy[v] += wl * ly;
                    } else {  // stage 1, q == 3: line-slope part of the accumulator
                        accs[(4 * l + v) * P + c] = dx_ * ridx;
                        accs[(4 * M + 4 * l + v) * P + c] = dy_ * ridy;
                    }
                }
            }
        }
        bool bad = false;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double Wn;
            if (BULK32) {
                // float-float: the exact differences of the face sums (two-sums),
                // the bases' flux differences times dt/2 or dt, over dx and dy;
                // one conversion to FP64 per quantity (the FP64 pipe is narrow)
                const ff ix = {g.idxf, g.idxlo}, iy = {g.idyf, g.idylo};
                ff tx = ff_two_sum((float)gxr0[v], -(float)gxl0[v]), ty = ff_two_sum((float)gyr0[v], -(float)gyl0[v]);
                if (STAGE == 1) {
                    const ff hdt = {0.5f * g.dtf[0], 0.5f * g.dtf[1]}, fdt = {g.dtf[0], g.dtf[1]};
                    tx = ff_add(tx, ff_mul(hdt, Bx[v]));
                    ty = ff_add(ty, ff_mul(hdt, By[v]));
                    ff ax = ff_add(ff_two_sum((float)gxr1[v], -(float)gxl1[v]), ff_mul(fdt, Bx[v]));
                    ff ay = ff_add(ff_two_sum((float)gyr1[v], -(float)gyl1[v]), ff_mul(fdt, By[v]));
                    double W = g.S0[v * P + c];
                    Wn = W - ff_val(ff_add(ff_mul(tx, ix), ff_mul(ty, iy)));  // Eq. 2.21
                    g.ACC[v * P + c] = W - ff_val(ff_add(ff_mul(ax, ix), ff_mul(ay, iy)));
                } else {
                    Wn = g.ACC[v * P + c] - ff_val(ff_add(ff_mul(tx, ix), ff_mul(ty, iy)));  // Eq. 2.22-2.23
                }
            } else {
                const double dx0 = exact_diff(gxr0[v], gxl0[v]), dy0 = exact_diff(gyr0[v], gyl0[v]);
                if (STAGE == 1) {
                    double W = g.S0[v * P + c];
                    Wn = W - dx0 * idx - dy0 * idy;  // Eq. 2.21
                    g.ACC[v * P + c] = W - exact_diff(gxr1[v], gxl1[v]) * idx - exact_diff(gyr1[v], gyl1[v]) * idy;
                } else {
                    Wn = g.ACC[v * P + c] - dx0 * idx - dy0 * idy;  // Eq. 2.22-2.23
                }
            }
            // the FP32-bulk stage 2 reads W* from the float planes only
            if (!BULK32 || STAGE == 2) out[v * P + c] = Wn;
            bad |= !isfinite(Wn);
            if (BULK32) {
                const float hi = (float)Wn;
                outf[v * P + c] = hi;
                outf[(12 + 8 * M + v) * P + c] = (float)(Wn - (double)hi);  // low part
                outf[(4 + v) * P + c] = (float)sx[v];  // cell slopes: Gauss sum of the line slopes
                outf[(8 + v) * P + c] = (float)sy[v];
            } else {
                out[(4 + v) * P + c] = (double)sx[v];
                out[(8 + v) * P + c] = (double)sy[v];
            }
        }
        // face sigma of this step (Eq. 3.1): mean over the face's Gauss points
        if (STAGE == 1) {
            const double* SX = g.SP[0];
            const double* SY = g.SP[1];
            double s = 0;
            for (int l = 0; l < M; ++l) s += SX[((long long)j * (g.nx + 1) + i) * M + l];
            g.sig_xn[(long long)j * (g.nx + 1) + i] = s / M;
            if (i == g.nx - 1) {
                s = 0;
                for (int l = 0; l < M; ++l) s += SX[((long long)j * (g.nx + 1) + g.nx) * M + l];
                g.sig_xn[(long long)j * (g.nx + 1) + g.nx] = s / M;
            }
            s = 0;
            for (int l = 0; l < M; ++l) s += SY[((long long)j * g.nx + i) * M + l];
            g.sig_yn[(long long)j * g.nx + i] = s / M;
            if (j == g.ny - 1) {
                s = 0;
                for (int l = 0; l < M; ++l) s += SY[((long long)g.ny * g.nx + i) * M + l];
                g.sig_yn[(long long)g.ny * g.nx + i] = s / M;
            }
        } else {
            g.sig_x[(long long)j * (g.nx + 1) + i] = g.sig_xn[(long long)j * (g.nx + 1) + i];
            if (i == g.nx - 1) g.sig_x[(long long)j * (g.nx + 1) + g.nx] = g.sig_xn[(long long)j * (g.nx + 1) + g.nx];
            g.sig_y[(long long)j * g.nx + i] = g.sig_yn[(long long)j * g.nx + i];
            if (j == g.ny - 1) g.sig_y[(long long)g.ny * g.nx + i] = g.sig_yn[(long long)g.ny * g.nx + i];
        }
        if (bad) flag_bad(g, c);
    }
}

// -------------------------------------------------------------- update (1-D)
template <typename R, int STAGE, bool ONE>
__global__ void __launch_bounds__(256) k_update1(Work w)
{
    constexpr bool BULK32 = sizeof(R) == 4;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        long long il;
        const Mesh& g = mesh_of<ONE>(w, gi, il);
        int i = (int)il;
        const R* FX = (const R*)g.FO[0];
        // q-th output quantity of variable v at face i (left) or i + 1 (right)
        const long long nf = g.nx + 1;
        auto xl = [&](int e) { return FX[fo_off(nf, 1, e >> 2, 0, i) + (e & 3)]; };
        auto xr = [&](int e) { return FX[fo_off(nf, 1, e >> 2, 0, i + 1) + (e & 3)]; };
        const double idx = g.idx;
        long long P = g.plane;
        bool bad = false;
        // FP32 bulk, stage 1: face outputs are increments over hi of the face's
        // right cell (i, and i+1); their flux parts add the float-float Euler
        // fluxes of the bases, their state parts the bases' difference
        double B[3] = {0, 0, 0}, hd[3] = {0, 0, 0};
        if (BULK32 && STAGE == 1) {
            const double tb = *g.tn;
            float h0[3], h1[3];
            for (int v = 0; v < 3; ++v) {
                h0[v] = g.F0[v * P + i];
                h1[v] = cell<1, 1, float, true>(g, g.F0, 0, v, 0, i + 1, 0, tb);
                hd[v] = (double)(h1[v] - h0[v]);
            }
            const double gm1d = g.gamma - 1.0;
            const ff gm1 = {(float)gm1d, (float)(gm1d - (double)(float)gm1d)};
            ff f0[3], f1[3];
            euler_flux_ff<1>(h0, gm1, f0);
            euler_flux_ff<1>(h1, gm1, f1);
            for (int v = 0; v < 3; ++v) B[v] = ff_val(ff_add(f1[v], ff_neg(f0[v])));
        }
        for (int v = 0; v < 3; ++v) {
            double Wn, Sn;
            if (STAGE == 1) {
                double W = g.S0[v * P + i];
                const double dtd = *g.dt;
                Wn = W - (((double)xr(v) - (double)xl(v)) + 0.5 * dtd * B[v]) * idx;
                Sn = (((double)xr(8 + v) - (double)xl(8 + v)) + hd[v]) * idx;
                if (!BULK32) g.S1[v * P + i] = Wn;  // the FP32-bulk stage 2 reads the float planes
                g.ACC[v * P + i] = W - (((double)xr(4 + v) - (double)xl(4 + v)) + dtd * B[v]) * idx;
                g.ACC[(3 + v) * P + i] = (((double)xr(12 + v) - (double)xl(12 + v)) + hd[v]) * idx;
            } else {
                Wn = g.ACC[v * P + i] - ((double)xr(v) - (double)xl(v)) * idx;
                Sn = g.ACC[(3 + v) * P + i] + ((double)xr(4 + v) - (double)xl(4 + v)) * idx;
                g.S0[v * P + i] = Wn;
            }
            if (BULK32) {
                float* outf = STAGE == 1 ? g.F1 : g.F0;
                const float hi = (float)Wn;
                outf[v * P + i] = hi;
                outf[(6 + v) * P + i] = (float)(Wn - (double)hi);  // low part
                outf[(3 + v) * P + i] = (float)Sn;
            } else {
                (STAGE == 1 ? g.S1 : g.S0)[(3 + v) * P + i] = Sn;
            }
            bad |= !isfinite(Wn);
        }
        if (STAGE == 1) {
            g.sig_xn[i] = g.SP[0][i];
            if (i == g.nx - 1) g.sig_xn[g.nx] = g.SP[0][g.nx];
        } else {
            g.sig_x[i] = g.sig_xn[i];
            if (i == g.nx - 1) g.sig_x[g.nx] = g.sig_xn[g.nx];
        }
        if (bad) flag_bad(g, i);
    }
}

// -------------------------------------------------------------- FP32-bulk state copies
// to_float: all FP64 planes of state n -> the float planes (after a state is set);
// otherwise the float slope planes -> the FP64 planes (before a state is read
// out; the FP64 cell averages are already current).
template <int D, int M>
__global__ void __launch_bounds__(256) k_convert(Work w, int to_float)
{
    constexpr int NP = D == 2 ? 12 + 8 * M : 6;
    constexpr int NV = D + 2;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        long long c = gi - w.off[k];
        long long P = g.plane;
        if (to_float) {
            for (int p = 0; p < NP; ++p) g.F0[p * P + c] = (float)g.S0[p * P + c];
            // low parts of the cell averages, after the other planes
            for (int v = 0; v < NV; ++v) g.F0[(NP + v) * P + c] = low_part<float>(g.S0[v * P + c]);
        } else {
            for (int p = NV; p < NP; ++p) g.S0[p * P + c] = (double)g.F0[p * P + c];
        }
    }
}

// -------------------------------------------------------------- CFL (Sec. 4)
// max over cells of (|U| + a) / h (and 4 nu / h^2 for viscous flow), h =
// min(dx, dy); one atomicMax per block on the
// bit pattern of a positive double (ordered like the value).  The plain form
// evaluates the speeds in FP64 from the FP64 averages; the FP32-bulk form in
// FP32 from its float state planes (the step size is not a conserved
// quantity: its 1e-7 relative rounding only shifts where the steps fall),
// and the maximum is taken in FP64 in both.
template <int D, typename R>
__global__ void __launch_bounds__(256) k_cfl(Work w)
{
    __shared__ double red[8];
    double best = 0.0;
    int kprev = -1;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        if (k != kprev && kprev >= 0 && best > 0.0)
            atomicMax(w.mesh[kprev].smax, (unsigned long long)__double_as_longlong(best)), best = 0.0;
        kprev = k;
        long long c = gi - w.off[k];
        long long P = g.plane;
        const R* S = state_planes<R>(g, 0);
        const R gm = MeshR<R>::gamma(g);
        R rho = S[c], ir = (R)1 / rho;
        R mu = S[P + c] * ir;
        R mv = D == 2 ? S[2 * P + c] * ir : (R)0;
        R E = S[(D + 1) * P + c];
        R q2 = mu * mu + mv * mv;
        R p = (gm - (R)1) * (E - (R)0.5 * rho * q2);
        R ih = D == 2 ? fmax(MeshR<R>::ih(g, 0), MeshR<R>::ih(g, 1)) : MeshR<R>::ih(g, 0);  // 1 / min(dx, dy)
        R sp = (sqrt(q2) + sqrt(gm * p * ir)) * ih;
        // viscous flow: the diffusive limit dt <= h^2 / (4 nu), nu = mu / rho
        if (g.tau_mode == 2) sp = fmax(sp, (R)4 * MeshR<R>::mu(g) * ir * ih * ih);
        double s = (double)sp;
        if (!(s == s)) s = 1e300;  // a NaN state yields a tiny step and is flagged by the stages
        best = fmax(best, s);
    }
    // single-mesh tables reduce per block; batches flush per mesh change above
    if (w.n == 1) {
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b = fmax(b, red[q]);
            if (b > 0.0) atomicMax(w.mesh[0].smax, (unsigned long long)__double_as_longlong(b));
        }
    } else if (kprev >= 0 && best > 0.0) {
        atomicMax(w.mesh[kprev].smax, (unsigned long long)__double_as_longlong(best));
    }
}

// dt = cfl / smax per mesh (or the fixed value); t^n = t, t += dt; reset the reduction
template <int Unused = 0>
__global__ void k_dt(Mesh* meshes, int n, int use_cfl, const double* fixed)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        Mesh& g = meshes[k];
        double dt;
        if (use_cfl) {
            double s = __longlong_as_double((long long)*g.smax);
            dt = s > 0.0 ? g.cfl / s : 0.0;
            *g.smax = 0ull;
        } else {
            dt = fixed[k];
        }
        *g.dt = dt;
        g.dtf[0] = (float)dt;
        g.dtf[1] = (float)(dt - (double)g.dtf[0]);
        *g.tn = *g.t;
        *g.t += dt;
        for (int q = 0; q < 4; ++q) g.branch[q] = 0ull;  // counts cover the latest step
    }
}

// initial sigma from the two cell averages adjacent to each face (Eq. 3.2)
template <int D>
__global__ void k_sigma_init(Work w)
{
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        long long li = gi - w.off[k];
        long long nxf = (long long)(g.nx + 1) * g.ny;
        int dir = li < nxf ? 0 : 1;
        if (dir == 1) li -= nxf;
        int f, b;
        if (dir == 0) { f = (int)(li % (g.nx + 1)); b = (int)(li / (g.nx + 1)); }
        else { b = (int)(li % g.nx); f = (int)(li / g.nx); }
        double Ws[2][4];
        const double tb = *g.t;  // inflow ghost states at the current time
        for (int s = 0; s < 2; ++s)
            for (int v = 0; v < D + 2; ++v) {
                int a = f - 1 + s;
                Ws[s][v] = dir == 0 ? cell<D, 4, double>(g, g.S0, 0, v, 0, a, b, tb)
                                    : cell<D, 4, double>(g, g.S0, 0, v, 0, b, a, tb);
            }
        double pz[2], mn[2], mt[2];
        for (int s = 0; s < 2; ++s) {
            double rho = Ws[s][0];
            double u = Ws[s][1] / rho, v = D == 2 ? Ws[s][2] / rho : 0.0;
            double p = (g.gamma - 1.0) * (Ws[s][D + 1] - 0.5 * rho * (u * u + v * v));
            double c = sqrt(g.gamma * p / rho);
            pz[s] = p;
            mn[s] = (dir == 0 ? u : v) / c;
            mt[s] = (dir == 0 ? v : u) / c;
        }
        double dp = fabs(pz[0] - pz[1]);
        double sig = dp / pz[0] + dp / pz[1] + (mn[0] - mn[1]) * (mn[0] - mn[1]) + (mt[0] - mt[1]) * (mt[0] - mt[1]);
        if (dir == 0) g.sig_x[(long long)b * (g.nx + 1) + f] = sig;
        else g.sig_y[(long long)f * g.nx + b] = sig;
    }
}

// positivity of a state set in (host-side check is done on the device)
template <int D>
__global__ void k_check_state(Work w)
{
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        long long c = gi - w.off[k];
        long long P = g.plane;
        double rho = g.S0[c], u = g.S0[P + c] / rho, v = D == 2 ? g.S0[2 * P + c] / rho : 0.0;
        double p = (g.gamma - 1.0) * (g.S0[(D + 1) * P + c] - 0.5 * rho * (u * u + v * v));
        if (!(rho > 0.0) || !(p > 0.0)) flag_bad(g, c);
    }
}

} // namespace cgks
