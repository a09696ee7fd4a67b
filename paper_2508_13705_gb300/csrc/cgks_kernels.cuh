// Stage kernels of the ASE-DFF-CGKS step.  See cgks_device.cuh for the
// mathematics; this file maps it onto grid-stride loops over the work items
// of every mesh in a descriptor table.
//
// Local frame of a direction: dir 0 (faces normal to x): a = i (normal
// index), b = j (tangential); dir 1 (faces normal to y): a = j, b = i.
// Momentum components are ordered normal first in the local frame.
//
// Scratch layouts per mesh and direction (na, nb: cells along / across the
// normal; M Gauss points per face):
//   LA  [nb+2][na+6][M][4]            line averages, b in [-1, nb], a in [-3, na+2]
//   FR  [nb+2][na+1][M][2][3][4]      face states: side 0 = left (from cell f-1),
//                                     side 1 = right (from cell f); W, W_n, W_nn
//   FO  [nb][na+1][M][16]             per-point stage outputs (global frame)
//   SP  [nb][na+1][M]                 sigma per face Gauss point (Eq. 3.2)
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

// cell value in local coordinates; lkind: 0 W, 1 W_n (cell), 2 W_t (cell), 3 W_n line
template <int D, int M>
__device__ __forceinline__ double lcell(const Mesh& g, const double* S, int dir, int lkind, int v, int l, int a, int b)
{
    int kind;
    if (lkind == 0) kind = 0;
    else if (lkind == 1) kind = dir == 0 ? 1 : 2;
    else if (lkind == 2) kind = dir == 0 ? 2 : 1;
    else kind = dir == 0 ? 3 : 4;
    int i = dir == 0 ? a : b, j = dir == 0 ? b : a;
    return cell<D, M>(g, S, kind, vglob(dir, v), l, i, j);
}

// sigma of normal faces (f, b) and of tangential faces of column a (a, f)
template <int D>
__device__ __forceinline__ double lsigN(const Mesh& g, const double* sx, const double* sy, int dir, int f, int b)
{
    return dir == 0 ? sigx<D>(g, sx, f, b) : sigy(g, sy, b, f);
}
__device__ __forceinline__ double lsigT(const Mesh& g, const double* sx, const double* sy, int dir, int a, int f)
{
    return dir == 0 ? sigy(g, sy, a, f) : sigx<2>(g, sx, f, a);
}

__device__ __forceinline__ void flag_bad(const Mesh& g, long long idx)
{
    atomicOr(g.status, STATUS_NONPHYS);
    atomicMin((unsigned long long*)g.bad, (unsigned long long)idx);
}

// -------------------------------------------------------------- Step 1 (2-D)
template <int M, typename R>
__global__ void __launch_bounds__(256) k_lines(Work w, int stage)
{
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        long long li = gi - w.off[k];
        long long nxl = (long long)(g.nx + 6) * (g.ny + 2);
        int dir = li < nxl ? 0 : 1;
        if (dir == 1) li -= nxl;
        int na, nb;
        local_dims<M>(g, dir, na, nb);
        int a = (int)(li % (na + 6)) - 3;
        int b = (int)(li / (na + 6)) - 1;
        const double* S = stage == 1 ? g.S0 : g.S1;
        double s6[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) s6[q] = lsigT(g, g.sig_x, g.sig_y, dir, a, b - 2 + q);
        Dff dff = dff_select(g.order, s6, g.thr);
        double ht = dir == 0 ? g.dy : g.dx;
        int rows[M];
#pragma unroll
        for (int l = 0; l < M; ++l) rows[l] = 6 + l;
        R* LA = (R*)g.LA[dir] + (((long long)(b + 1) * (na + 6) + (a + 3)) * M) * 4;
#pragma unroll 1
        for (int v = 0; v < 4; ++v) {
            double qi = lcell<2, M>(g, S, dir, 0, v, 0, a, b);
            R dp[10];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                dp[q] = (R)(lcell<2, M>(g, S, dir, 0, v, 0, a, b + q - 2) - qi);
                dp[5 + q] = (R)(ht * lcell<2, M>(g, S, dir, 2, v, 0, a, b + q - 2));
            }
            R out[M];
            recon<R, M>(dff, g.oi, rows, 0, dp, out, g.ghi, g.glo, g.eps);
#pragma unroll
            for (int l = 0; l < M; ++l) LA[l * 4 + v] = (R)(qi + (double)out[l]);
        }
    }
}

// -------------------------------------------------------------- Step 2
// D == 1: the cell data are the cell averages and slopes themselves.
template <int D, int M, typename R>
__global__ void __launch_bounds__(256) k_normal(Work w, int stage)
{
    __shared__ unsigned long long cnt[4];
    if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        long long li = gi - w.off[k];
        int dir = 0, na = g.nx, nb = 1;
        if (D == 2) {
            long long nxl = (long long)(g.nx + 2) * (g.ny + 2) * M;
            dir = li < nxl ? 0 : 1;
            if (dir == 1) li -= nxl;
            local_dims<M>(g, dir, na, nb);
        }
        int l = D == 2 ? (int)(li % M) : 0;
        long long r = D == 2 ? li / M : li;
        int a = (int)(r % (na + 2)) - 1;
        int b = D == 2 ? (int)(r / (na + 2)) - 1 : 0;
        const double* S = stage == 1 ? g.S0 : g.S1;
        double s6[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) s6[q] = D == 2 ? lsigN<2>(g, g.sig_x, g.sig_y, dir, a - 2 + q, b)
                                                   : sigx<1>(g, g.sig_x, a - 2 + q, 0);
        Dff dff = dff_select(g.order, s6, g.thr);
        {
            int bi = dff.st < 0 ? 0 : dff.st - ST_R5 + 1;
            atomicAdd(&cnt[bi], 1ull);
        }
        double hn = dir == 0 ? g.dx : g.dy;
        const int rows[6] = {0, 1, 2, 3, 4, 5};
        const R* LA = D == 2 ? (const R*)g.LA[dir] : nullptr;
        R* FR = (R*)g.FR[dir];
        constexpr int NV = D + 2;
#pragma unroll 1
        for (int v = 0; v < NV; ++v) {
            double qi;
            R dp[10];
            if (D == 2) {
                const R* la = LA + ((long long)(b + 1) * (na + 6) + (a + 3)) * M * 4 + l * 4 + v;
                qi = (double)la[0];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    dp[q] = (R)((double)la[(q - 2) * M * 4] - qi);
                    dp[5 + q] = (R)(hn * lcell<2, M>(g, S, dir, 3, v, l, a + q - 2, b));
                }
            } else {
                qi = cell<1, 1>(g, S, 0, v, 0, a, 0);
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    dp[q] = (R)(cell<1, 1>(g, S, 0, v, 0, a + q - 2, 0) - qi);
                    dp[5 + q] = (R)(hn * cell<1, 1>(g, S, 1, v, 0, a + q - 2, 0));
                }
            }
            R out[6];
            recon<R, 6>(dff, g.oi, rows, 0, dp, out, g.ghi, g.glo, g.eps);
            R ih = (R)(1.0 / hn);
            // side 0: left state of face a+1 (value at xi = +1/2)
            if (a + 1 <= na) {
                R* fr = FR + ((((long long)(b + 1) * (na + 1) + (a + 1)) * M + l) * 2 + 0) * 3 * 4;
                fr[0 * 4 + v] = (R)(qi + (double)out[0]);
                fr[1 * 4 + v] = out[1] * ih;
                fr[2 * 4 + v] = out[2] * ih * ih;
            }
            // side 1: right state of face a (value at xi = -1/2)
            if (a >= 0) {
                R* fr = FR + ((((long long)(b + 1) * (na + 1) + a) * M + l) * 2 + 1) * 3 * 4;
                fr[0 * 4 + v] = (R)(qi + (double)out[3]);
                fr[1 * 4 + v] = out[4] * ih;
                fr[2 * 4 + v] = out[5] * ih * ih;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 4 && cnt[threadIdx.x] && w.n > 0) atomicAdd(&w.mesh[0].branch[threadIdx.x], cnt[threadIdx.x]);
}

// -------------------------------------------------------------- Step 3 + flux
template <int D, int M, typename R, int STAGE>
__global__ void __launch_bounds__(128) k_flux(Work w)
{
    constexpr int NV = D + 2;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        long long li = gi - w.off[k];
        int dir = 0, na = g.nx, nb = 1;
        if (D == 2) {
            long long nxl = (long long)(g.nx + 1) * g.ny * M;
            dir = li < nxl ? 0 : 1;
            if (dir == 1) li -= nxl;
            local_dims<M>(g, dir, na, nb);
        }
        int l = D == 2 ? (int)(li % M) : 0;
        long long r = D == 2 ? li / M : li;
        int f = (int)(r % (na + 1));
        int b = D == 2 ? (int)(r / (na + 1)) : 0;
        const R* FR = (const R*)g.FR[dir];
        SideData<R, D> sd[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const R* fr = FR + ((((long long)(b + 1) * (na + 1) + f) * M + l) * 2 + side) * 12;
#pragma unroll
            for (int nd = 0; nd < 3; ++nd)
#pragma unroll
                for (int v = 0; v < 4; ++v) sd[side].d[nd][v] = v < NV ? fr[nd * 4 + v] : (R)0;
            if (D == 2) {
                // Step 3: tangential derivatives from the 3M face points of
                // segments b-1, b, b+1, scaled by the tangential r5 DFF of the
                // reconstructing cell (a = f-1 for the left state, f for the right)
                int a = side == 0 ? f - 1 : f;
                double s6[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) s6[q] = lsigT(g, g.sig_x, g.sig_y, dir, a, b - 2 + q);
                double at = dff_alpha(s6[1] + s6[2] + s6[3] + s6[4], g.thr);
                double ht = dir == 0 ? g.dy : g.dx;
                const auto& T = Tab<R>::get(g.oi);
                R c1 = (R)(at / ht), c2 = (R)(at / (ht * ht));
                R wt[4] = {0, 0, 0, 0}, wtt[4] = {0, 0, 0, 0}, wnt[4] = {0, 0, 0, 0};
#pragma unroll
                for (int s = 0; s < 3; ++s)
#pragma unroll
                    for (int kk = 0; kk < M; ++kk) {
                        const R* q = FR + ((((long long)(b + s) * (na + 1) + f) * M + kk) * 2 + side) * 12;
                        R w1 = T.d1[l][s * M + kk], w2 = T.d2[l][s * M + kk];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            R x0 = q[v], x1 = q[4 + v];
                            wt[v] += w1 * x0;
                            wtt[v] += w2 * x0;
                            wnt[v] += w1 * x1;
                        }
                    }
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    sd[side].d[3][v] = c1 * wt[v];
                    sd[side].d[4][v] = c2 * wtt[v];
                    sd[side].d[5][v] = c1 * wnt[v];
                }
            }
        }
        // Eq. 3.2 sigma and positivity of the reconstructed states in FP64
        double pz[2], mn[2], mt[2];
        bool bad = false;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            double rho = (double)sd[side].d[0][0];
            double un = (double)sd[side].d[0][1] / rho;
            double ut = D == 2 ? (double)sd[side].d[0][2] / rho : 0.0;
            double p = (g.gamma - 1.0) * ((double)sd[side].d[0][NV - 1] - 0.5 * rho * (un * un + ut * ut));
            double c = sqrt(g.gamma * p / rho);
            pz[side] = p; mn[side] = un / c; mt[side] = ut / c;
            bad |= !(rho > 0.0) || !(p > 0.0);
        }
        double dpz = fabs(pz[0] - pz[1]);
        double sig = dpz / pz[0] + dpz / pz[1] + (mn[0] - mn[1]) * (mn[0] - mn[1]) + (mt[0] - mt[1]) * (mt[0] - mt[1]);
        double dt = *g.dt;
        R F[4], Ft[4], Q0[4], Wt[4], Wtt[4];
        bool ok = kinetic<R, D>(sd[0], sd[1], (R)g.gamma, (R)g.K, g.tau_mode, (R)g.c1, (R)g.c2, (R)dt, F, Ft, Q0, Wt, Wtt);
        long long pt = (((long long)b * (na + 1) + f) * M + l);
        R* FO = (R*)g.FO[dir] + pt * 16;
        R Dt = (R)dt;
        bool finite = true;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            int gv = D == 2 ? vglob(dir, v) : v;
            if (STAGE == 1) {
                R o0 = (R)0.5 * Dt * F[v] + (R)0.125 * Dt * Dt * Ft[v];
                R o1 = Dt * F[v] + Dt * Dt / (R)6 * Ft[v];
                R o2 = Q0[v] + (R)0.5 * Dt * Wt[v] + (R)0.125 * Dt * Dt * Wtt[v];
                R o3 = Q0[v] + Dt * Wt[v] + Dt * Dt / (R)6 * Wtt[v];
                FO[0 * 4 + gv] = o0; FO[1 * 4 + gv] = o1; FO[2 * 4 + gv] = o2; FO[3 * 4 + gv] = o3;
                finite &= isfinite((double)o0) && isfinite((double)o1) && isfinite((double)o2) && isfinite((double)o3);
            } else {
                R o0 = Dt * Dt / (R)3 * Ft[v];
                R o1 = Dt * Dt / (R)3 * Wtt[v];
                FO[0 * 4 + gv] = o0; FO[1 * 4 + gv] = o1;
                finite &= isfinite((double)o0) && isfinite((double)o1);
            }
        }
        if (STAGE == 1) g.SP[dir][pt] = sig;
        if (bad || !ok || !finite) flag_bad(g, pt);
    }
}

// -------------------------------------------------------------- update (2-D)
template <int M, typename R, int STAGE>
__global__ void __launch_bounds__(256) k_update2(Work w)
{
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        long long c = gi - w.off[k];
        int i = (int)(c % g.nx), j = (int)(c / g.nx);
        const auto& T = Tab<double>::get(g.oi);
        const R* FX = (const R*)g.FO[0];
        const R* FY = (const R*)g.FO[1];
        // x-faces: b = j, f = i and i+1; y-faces: b = i, f = j and j+1
        const R* xl = FX + (((long long)j * (g.nx + 1) + i) * M) * 16;
        const R* xr = xl + M * 16;
        const R* yl = FY + (((long long)i * (g.ny + 1) + j) * M) * 16;
        const R* yr = yl + M * 16;
        double idx = 1.0 / g.dx, idy = 1.0 / g.dy;
        long long P = g.plane;
        double* out = STAGE == 1 ? g.S1 : g.S0;
        const double* Sin = g.S0;
        bool bad = false;
#pragma unroll 1
        for (int v = 0; v < 4; ++v) {
            double fx0 = 0, fy0 = 0, fx1 = 0, fy1 = 0;
            double sx = 0, sy = 0;
#pragma unroll
            for (int l = 0; l < M; ++l) {
                double wl = T.gw[l];
                fx0 += wl * ((double)xr[l * 16 + v] - (double)xl[l * 16 + v]);
                fy0 += wl * ((double)yr[l * 16 + v] - (double)yl[l * 16 + v]);
                if (STAGE == 1) {
                    fx1 += wl * ((double)xr[l * 16 + 4 + v] - (double)xl[l * 16 + 4 + v]);
                    fy1 += wl * ((double)yr[l * 16 + 4 + v] - (double)yl[l * 16 + 4 + v]);
                    double lx = ((double)xr[l * 16 + 8 + v] - (double)xl[l * 16 + 8 + v]) * idx;
                    double ly = ((double)yr[l * 16 + 8 + v] - (double)yl[l * 16 + 8 + v]) * idy;
                    out[(12 + 4 * l + v) * P + c] = lx;
                    out[(12 + 4 * M + 4 * l + v) * P + c] = ly;
                    sx += wl * lx;
                    sy += wl * ly;
                    g.ACC[(4 + 4 * l + v) * P + c] = ((double)xr[l * 16 + 12 + v] - (double)xl[l * 16 + 12 + v]) * idx;
                    g.ACC[(4 + 4 * M + 4 * l + v) * P + c] = ((double)yr[l * 16 + 12 + v] - (double)yl[l * 16 + 12 + v]) * idy;
                } else {
                    double lx = g.ACC[(4 + 4 * l + v) * P + c] + ((double)xr[l * 16 + 4 + v] - (double)xl[l * 16 + 4 + v]) * idx;
                    double ly = g.ACC[(4 + 4 * M + 4 * l + v) * P + c] + ((double)yr[l * 16 + 4 + v] - (double)yl[l * 16 + 4 + v]) * idy;
                    out[(12 + 4 * l + v) * P + c] = lx;
                    out[(12 + 4 * M + 4 * l + v) * P + c] = ly;
                    sx += wl * lx;
                    sy += wl * ly;
                }
            }
            if (STAGE == 1) {
                double W = Sin[v * P + c];
                double Ws = W - fx0 * idx - fy0 * idy;   // Eq. 2.21
                out[v * P + c] = Ws;
                g.ACC[v * P + c] = W - fx1 * idx - fy1 * idy;
                bad |= !isfinite(Ws);
            } else {
                double Wn = g.ACC[v * P + c] - fx0 * idx - fy0 * idy;  // Eq. 2.22-2.23
                out[v * P + c] = Wn;
                bad |= !isfinite(Wn);
            }
            out[(4 + v) * P + c] = sx;   // cell slopes: Gauss sum of the line slopes
            out[(8 + v) * P + c] = sy;
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
            for (int l = 0; l < M; ++l) s += SY[((long long)i * (g.ny + 1) + j) * M + l];
            g.sig_yn[(long long)j * g.nx + i] = s / M;
            if (j == g.ny - 1) {
                s = 0;
                for (int l = 0; l < M; ++l) s += SY[((long long)i * (g.ny + 1) + g.ny) * M + l];
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
template <typename R, int STAGE>
__global__ void __launch_bounds__(256) k_update1(Work w)
{
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < w.total;
         gi += (long long)gridDim.x * blockDim.x) {
        int k = find_mesh(w, gi);
        const Mesh& g = w.mesh[k];
        int i = (int)(gi - w.off[k]);
        const R* FX = (const R*)g.FO[0];
        const R* xl = FX + (long long)i * 16;
        const R* xr = xl + 16;
        double idx = 1.0 / g.dx;
        long long P = g.plane;
        bool bad = false;
        for (int v = 0; v < 3; ++v) {
            if (STAGE == 1) {
                double W = g.S0[v * P + i];
                double Ws = W - ((double)xr[v] - (double)xl[v]) * idx;
                g.S1[v * P + i] = Ws;
                g.S1[(3 + v) * P + i] = ((double)xr[8 + v] - (double)xl[8 + v]) * idx;
                g.ACC[v * P + i] = W - ((double)xr[4 + v] - (double)xl[4 + v]) * idx;
                g.ACC[(3 + v) * P + i] = ((double)xr[12 + v] - (double)xl[12 + v]) * idx;
                bad |= !isfinite(Ws);
            } else {
                double Wn = g.ACC[v * P + i] - ((double)xr[v] - (double)xl[v]) * idx;
                g.S0[v * P + i] = Wn;
                g.S0[(3 + v) * P + i] = g.ACC[(3 + v) * P + i] + ((double)xr[4 + v] - (double)xl[4 + v]) * idx;
                bad |= !isfinite(Wn);
            }
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

// -------------------------------------------------------------- CFL (Sec. 4)
// max over cells of (|U| + a) / min(dx, dy); one atomicMax per block on the
// bit pattern of a positive double (ordered like the value).
template <int D>
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
        double rho = g.S0[c], mu = g.S0[P + c] / rho;
        double mv = D == 2 ? g.S0[2 * P + c] / rho : 0.0;
        double E = g.S0[(D + 1) * P + c];
        double p = (g.gamma - 1.0) * (E - 0.5 * rho * (mu * mu + mv * mv));
        double h = D == 2 ? fmin(g.dx, g.dy) : g.dx;
        double s = (sqrt(mu * mu + mv * mv) + sqrt(g.gamma * p / rho)) / h;
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

// dt = cfl / smax per mesh (or the fixed value); t += dt; reset the reduction
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
        for (int s = 0; s < 2; ++s)
            for (int v = 0; v < D + 2; ++v) {
                int a = f - 1 + s;
                Ws[s][v] = dir == 0 ? cell<D, 4>(g, g.S0, 0, v, 0, a, b) : cell<D, 4>(g, g.S0, 0, v, 0, b, a);
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
