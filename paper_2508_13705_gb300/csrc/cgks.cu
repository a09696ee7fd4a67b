// Host side of the C ABI declared in include/cgks.h.
//
// A single-mesh solver is a batch of one: every kernel is a grid-stride loop
// over the work items of all meshes of a descriptor table (see
// cgks_kernels.cuh), launched with one persistent grid sized to the GPU
// (SM count x resident blocks).  One S2O4 step (Sec. 2.2) is captured once as
// a CUDA graph:
//   [CFL reduction] -> dt -> stage 1 (lines, normal, flux, update)
//                         -> stage 2 (lines, normal, flux, update)
// Device memory of all meshes lives in one slab allocated at init.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/cgks.h"
#include "cgks_kernels.cuh"
#include "kfns.h"
#include "tables.h"

using namespace cgks;

namespace {

int g_tables_device = -1;  // device whose constant tables are loaded
std::mutex g_tables_mu;     // first uses from several host threads load the tables once

int load_tables()
{
    std::lock_guard<std::mutex> lock(g_tables_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CGKS_ECUDA;
    if (g_tables_device == dev) return CGKS_OK;
    CgksTables t[3];
    TabF f[3];
    for (int k = 0; k < 3; ++k) {
        if (cgks_build_tables(5 + 2 * k, &t[k]) != 0) return CGKS_EINVAL;
        for (int a = 0; a < 6; ++a)
            for (int b = 0; b < 10; ++b)
                for (int c = 0; c < 10; ++c) f[k].row[a][b][c] = (float)t[k].row[a][b][c];
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 5; ++b)
                for (int c = 0; c < 10; ++c) f[k].cpoly[a][b][c] = (float)t[k].cpoly[a][b][c];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) f[k].bm2[a][b] = (float)t[k].bm2[a][b];
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) f[k].bm4[a][b] = (float)t[k].bm4[a][b];
        for (int a = 0; a < 4; ++a) {
            f[k].gx[a] = (float)t[k].gx[a];
            f[k].gw[a] = (float)t[k].gw[a];
            for (int b = 0; b < 12; ++b) { f[k].d1[a][b] = (float)t[k].d1[a][b]; f[k].d2[a][b] = (float)t[k].d2[a][b]; }
        }
    }
    // one upload per translation unit (its constant tables serve both kernel sets)
    Kfns all[8] = {kfns_1_1_d(true), kfns_1_1_f(true), kfns_2_2_d(true), kfns_2_3_d(true), kfns_2_4_d(true),
                   kfns_2_2_f(true), kfns_2_3_f(true), kfns_2_4_f(true)};
    for (int q = 0; q < 8; ++q)
        if (all[q].upload(t, f) != 0) return CGKS_ECUDA;
    g_tables_device = dev;
    return CGKS_OK;
}

Kfns pick_kfns(int dim, int order, int prec, int tau_mode, const int bc[4], int pt_fallback, bool one)
{
    int M = (order - 1) / 2;
    Kfns k;
    if (dim == 1) k = prec == CGKS_FP64 ? kfns_1_1_d(one) : kfns_1_1_f(one);
    else if (prec == CGKS_FP64) k = M == 2 ? kfns_2_2_d(one) : (M == 3 ? kfns_2_3_d(one) : kfns_2_4_d(one));
    else k = M == 2 ? kfns_2_2_f(one) : (M == 3 ? kfns_2_3_f(one) : kfns_2_4_f(one));
    // the flux instances of the mesh's collision-time mode
    if (tau_mode == CGKS_TAU_HGKS || tau_mode == CGKS_TAU_NS)
        for (int c = 0; c < 2; ++c) { k.flux1v[c] = k.flux1h[c]; k.flux2v[c] = k.flux2h[c]; }
    // the point fallback has one instance (tau > 0, uncapped)
    if (pt_fallback == CGKS_PT_FALLBACK_FIRST_ORDER)
        for (int c = 0; c < 2; ++c) { k.flux1v[c] = k.flux1p; k.flux2v[c] = k.flux2p; }
    k.flux1 = k.flux1v[0];
    k.flux2 = k.flux2v[0];
    // stencil kernels with the wall ghost rules only where a side is a wall
    bool walls = false;
    for (int s = 0; s < (dim == 2 ? 4 : 2); ++s) walls = walls || bc[s] >= CGKS_BC_REFLECTIVE;
    if (walls) { k.recon[0] = k.reconw[0]; k.recon[1] = k.reconw[1]; k.normal = k.normalw; }
    return k;
}

// Work lists: tiles of the 2-D Steps 1-2 per direction (their counts follow
// the tile shape of each direction), 1-D cells of Step 2, face points, cells,
// faces.
enum { W_TILE0 = 0, W_TILE1, W_NORMAL, W_FLUX, W_CELLS, W_SIGINIT, W_COUNT };

// Tile shapes (cells along the normal x across it) the autotuner tries for
// the 2-D Steps 1-2; the first is the default.
const int kTileShapes[][2] = {{28, 8}, {60, 4}, {12, 16}, {28, 4}, {12, 8}, {124, 2}};
const int kNumTileShapes = 6;

} // namespace

struct cgks_batch {
    cgks_params p;
    int n = 0, dim = 2, M = 1, nvar = 4, nplanes = 0, nacc = 0;
    size_t rsize = 8;
    cudaStream_t stream = nullptr;
    std::vector<Mesh> host;      // host copy of the descriptors
    Mesh* dmesh = nullptr;       // device descriptors
    long long* doff = nullptr;   // device prefix arrays [W_COUNT][n+1]
    long long* doff1 = nullptr;  // per-mesh single-mesh tables [n][W_COUNT][2] = {0, items}
    std::vector<long long> off;  // host prefix arrays
    double* dfixed = nullptr;    // fixed dt per mesh
    char* slab = nullptr;
    Kfns k;
    int grid[16];
    int threads[16];  // threads per block of each kernel slot (autotuned)
    int tile[2][2];   // 2-D Steps 1-2: tile shape (TA, TB) per direction (autotuned)
    int nsm = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // [0] fixed dt, [1] CFL dt
    int kernels_per_step = 0;
    bool state_set = false;
    bool own_stream = false;
    bool sigma_pending = false;  // sigma was initialised by set_state and no step has run since
};

struct cgks_solver {
    cgks_batch* b = nullptr;
};

namespace {

#define CK(x)                                                   \
    do {                                                        \
        cudaError_t e_ = (x);                                   \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? CGKS_ENOMEM : CGKS_ECUDA; \
    } while (0)

Work work_of(const cgks_batch* b, int kind)
{
    Work w;
    w.mesh = b->dmesh;
    w.m0 = b->host[0];
    w.off = b->doff + (size_t)kind * (b->n + 1);
    w.n = b->n;
    w.total = b->off[(size_t)kind * (b->n + 1) + b->n];
    return w;
}

// Tiles of TA x TB cells covering a in [-1, na], b in [-1, nb] of direction dir.
long long tiles(int dir, int nx, int ny, int TA, int TB)
{
    long long na = dir == 0 ? nx : ny, nb = dir == 0 ? ny : nx;
    return ((na + 2 + TA - 1) / TA) * ((nb + 2 + TB - 1) / TB);
}

long long items(int kind, int dim, int M, int nx, int ny)
{
    (void)M;
    switch (kind) {
    case W_TILE0: return dim == 2 ? tiles(0, nx, ny, kTileShapes[0][0], kTileShapes[0][1]) : 0;
    case W_TILE1: return dim == 2 ? tiles(1, nx, ny, kTileShapes[0][0], kTileShapes[0][1]) : 0;
    case W_NORMAL: return dim == 2 ? 0 : nx + 2;
    case W_FLUX: return dim == 2 ? ((long long)(nx + 1) * ny + (long long)(ny + 1) * nx) * M : nx + 1;
    case W_CELLS: return (long long)nx * ny;
    default: return dim == 2 ? (long long)(nx + 1) * ny + (long long)(ny + 1) * nx : nx + 1;
    }
}

int launch(cgks_batch* b, const void* fn, int kind, int gi, int stage, bool has_stage)
{
    Work w = work_of(b, kind);
    if (w.total == 0) return CGKS_OK;
    int threads = b->threads[gi];
    long long need = (w.total + threads - 1) / threads;
    int grid = (int)std::min<long long>(need, (long long)b->grid[gi]);
    if (grid < 1) grid = 1;
    void* args2[] = {&w, &stage};
    void* args1[] = {&w};
    CK(cudaLaunchKernel(fn, dim3(grid), dim3(threads), has_stage ? args2 : args1, 0, b->stream));
    return CGKS_OK;
}

// Dynamic shared memory of the 2-D Steps 1-2 for a tile shape.
size_t recon_smem(const cgks_batch* b, int TA, int TB)
{
    return (size_t)(TA + 4) * TB * (4 * b->M + 8) * b->rsize;
}

// Set the tile shape of direction dir: the per-mesh tile counts of the work
// list (host and device), the kernel's shared-memory limit and its persistent
// grid at `threads` threads per block (slot dir).
int set_tile(cgks_batch* b, int dir, int TA, int TB, int threads)
{
    const void* fn = (const void*)b->k.recon[dir];
    size_t smem = recon_smem(b, TA, TB);
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1)
        return CGKS_ENOTSUP;
    b->tile[dir][0] = TA;
    b->tile[dir][1] = TB;
    b->threads[dir] = threads;
    b->grid[dir] = occ * b->nsm;
    const int kind = dir == 0 ? W_TILE0 : W_TILE1;
    long long* o = b->off.data() + (size_t)kind * (b->n + 1);
    o[0] = 0;
    for (int k = 0; k < b->n; ++k) o[k + 1] = o[k] + tiles(dir, b->host[k].nx, b->host[k].ny, TA, TB);
    CK(cudaMemcpy(b->doff + (size_t)kind * (b->n + 1), o, (b->n + 1) * sizeof(long long), cudaMemcpyHostToDevice));
    return CGKS_OK;
}

// One launch of the 2-D Steps 1-2 of direction dir (tiles as work items).
int launch_recon(cgks_batch* b, int dir, int stage)
{
    Work w = work_of(b, dir == 0 ? W_TILE0 : W_TILE1);
    if (w.total == 0) return CGKS_OK;
    int TA = b->tile[dir][0], TB = b->tile[dir][1];
    int grid = (int)std::max<long long>(1, std::min<long long>(w.total, (long long)b->grid[dir]));
    void* args[] = {&w, &stage, &TA, &TB};
    CK(cudaLaunchKernel((const void*)b->k.recon[dir], dim3(grid), dim3(b->threads[dir]), args,
                        recon_smem(b, TA, TB), b->stream));
    return CGKS_OK;
}

int enqueue_stage(cgks_batch* b, int stage)
{
    int r;
    if (b->dim == 2) {
        if ((r = launch_recon(b, 0, stage))) return r;
        if ((r = launch_recon(b, 1, stage))) return r;
    } else if ((r = launch(b, (const void*)b->k.normal, W_NORMAL, 1, stage, true))) {
        return r;
    }
    if ((r = launch(b, (const void*)(stage == 1 ? b->k.flux1 : b->k.flux2), W_FLUX, stage == 1 ? 2 : 3, 0, false))) return r;
    if ((r = launch(b, (const void*)(stage == 1 ? b->k.upd1 : b->k.upd2), W_CELLS, stage == 1 ? 4 : 5, 0, false))) return r;
    return CGKS_OK;
}

int enqueue_step(cgks_batch* b, bool cfl)
{
    int r;
    if (cfl && (r = launch(b, (const void*)b->k.cfl, W_CELLS, 6, 0, false))) return r;
    int use = cfl ? 1 : 0;
    const double* fx = b->dfixed;
    Mesh* dm = b->dmesh;
    int n = b->n;
    void* args[] = {&dm, &n, &use, &fx};
    CK(cudaLaunchKernel((const void*)k_dt<0>, dim3((n + 127) / 128), dim3(128), args, 0, b->stream));
    if ((r = enqueue_stage(b, 1))) return r;
    if ((r = enqueue_stage(b, 2))) return r;
    return CGKS_OK;
}

int build_graph(cgks_batch* b, int which)
{
    if (b->gexec[which]) return CGKS_OK;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int r = enqueue_step(b, which == 1);
    cudaGraph_t gg = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &gg);
    if (r) { if (gg) cudaGraphDestroy(gg); return r; }
    if (e != cudaSuccess) return CGKS_ECUDA;
    g = gg;
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    b->kernels_per_step = (int)nn;
    e = cudaGraphInstantiate(&b->gexec[which], g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? CGKS_OK : CGKS_ECUDA;
}

int validate(const cgks_params* p)
{
    if (!p) return CGKS_EINVAL;
    if (p->dim != 1 && p->dim != 2) return CGKS_EINVAL;
    if (p->order != 5 && p->order != 7 && p->order != 9) return CGKS_EINVAL;
    if (p->precision != CGKS_FP64 && p->precision != CGKS_FP32_BULK) return CGKS_EINVAL;
    if (p->tau_mode != CGKS_TAU_ZERO && p->tau_mode != CGKS_TAU_HGKS && p->tau_mode != CGKS_TAU_NS)
        return CGKS_EINVAL;
    if (!(p->mu >= 0.0) || !std::isfinite(p->mu) || (p->tau_mode == CGKS_TAU_NS && !(p->mu > 0.0)))
        return CGKS_EINVAL;
    if (p->dff_lag != CGKS_DFF_LAG_STEP && p->dff_lag != CGKS_DFF_LAG_STAGE) return CGKS_EINVAL;
    if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->sigma_thres > 0.0)) return CGKS_EINVAL;
    if (!(p->gamma_hi > 0.0 && p->gamma_hi < 1.0) || !(p->gamma_lo > 0.0 && p->gamma_lo < 1.0)) return CGKS_EINVAL;
    if (!(p->weno_eps > 0.0)) return CGKS_EINVAL;
    if (p->pt_fallback != CGKS_PT_FALLBACK_OFF && p->pt_fallback != CGKS_PT_FALLBACK_FIRST_ORDER) return CGKS_EINVAL;
    for (int s = 0; s < 4; ++s) {
        if (p->bc[s] < 0 || p->bc[s] > CGKS_BC_INFLOW_REFLECTIVE) return CGKS_EINVAL;
        if (p->bc[s] == CGKS_BC_FIXED && (p->dim == 2 || s >= 2)) return CGKS_EINVAL;
        if (p->bc[s] == CGKS_BC_INFLOW || p->bc[s] == CGKS_BC_INFLOW_REFLECTIVE) {
            if (p->dim != 2) return CGKS_EINVAL;
            if (!std::isfinite(p->bc_split[s][0]) || !std::isfinite(p->bc_split[s][1])) return CGKS_EINVAL;
            for (int h = 0; h < 2; ++h) {
                const double* q = p->bc_state[s][h];
                double rho = q[0];
                if (!(rho > 0.0) || !std::isfinite(rho)) return CGKS_EINVAL;
                double pr = (p->gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / rho);
                if (!(pr > 0.0) || !std::isfinite(pr)) return CGKS_EINVAL;
            }
        }
    }
    // the fallback is compiled into the collision-time (tau > 0) flux only
    if (p->pt_fallback && p->tau_mode == CGKS_TAU_ZERO) return CGKS_ENOTSUP;
    return CGKS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// per-mesh slab layout
struct Layout {
    size_t S, F, ACC, sigx, sigy, FR[2], FO[2], SP[2], AT[2], TD[2], scal, total;
};

Layout layout(int dim, int M, size_t rs, int nx, int ny)
{
    Layout L;
    size_t plane = (size_t)nx * ny;
    int np = dim == 2 ? 12 + 8 * M : 6;
    int nacc = dim == 2 ? 4 + 8 * M : 6;
    int nv = dim + 2;
    size_t o = 0;
    L.S = o; o = align256(o + 2 * np * plane * 8);
    // FP32-bulk float planes: every state plane plus the low parts of the averages
    L.F = o; o = align256(o + (rs == 4 ? 2 * (np + nv) * plane * 4 : 0));
    L.ACC = o; o = align256(o + nacc * plane * 8);
    L.sigx = o; o = align256(o + 2 * (size_t)(nx + 1) * ny * 8);
    L.sigy = o; o = align256(o + (dim == 2 ? 2 * (size_t)(ny + 1) * nx * 8 : 0));
    for (int d = 0; d < 2; ++d) {
        int na = d == 0 ? nx : ny, nb = d == 0 ? ny : nx;
        bool on = dim == 2 || d == 0;
        L.FR[d] = o; o = align256(o + (on ? (size_t)(nb + 2) * (na + 1) * M * 24 * rs : 0));
        L.FO[d] = o; o = align256(o + (on ? (size_t)nb * (na + 1) * M * 16 * rs : 0));
        L.SP[d] = o; o = align256(o + (on ? (size_t)nb * (na + 1) * M * 8 : 0));
        L.AT[d] = o; o = align256(o + (on && dim == 2 ? (size_t)(nb + 2) * (na + 6) * rs : 0));
        // FP32 bulk: each cell's tangential differences of hi, for Step 3
        L.TD[d] = o; o = align256(o + (on && dim == 2 && rs == 4 ? (size_t)(nb + 2) * (na + 6) * 8 * rs : 0));
    }
    L.scal = o; o = align256(o + 512);
    L.total = o;
    return L;
}

int batch_create(cgks_batch** out, const cgks_params* p, int n, const int* nx, const int* ny,
                 const double* ext, void* stream)
{
    if (!out) return CGKS_EINVAL;
    *out = nullptr;
    int r = validate(p);
    if (r) return r;
    if (n < 1 || !nx || !ny || !ext) return CGKS_EINVAL;
    for (int k = 0; k < n; ++k) {
        if (nx[k] < 1 || ny[k] < 1 || (p->dim == 1 && ny[k] != 1)) return CGKS_EINVAL;
        if (!(ext[4 * k + 1] > ext[4 * k]) || (p->dim == 2 && !(ext[4 * k + 3] > ext[4 * k + 2]))) return CGKS_EINVAL;
        // a wall mirrors up to 3 ghost layers onto distinct interior cells
        bool wx = p->bc[0] >= CGKS_BC_REFLECTIVE || p->bc[1] >= CGKS_BC_REFLECTIVE;
        bool wy = p->dim == 2 && (p->bc[2] >= CGKS_BC_REFLECTIVE || p->bc[3] >= CGKS_BC_REFLECTIVE);
        if ((wx && nx[k] < 3) || (wy && ny[k] < 3)) return CGKS_EINVAL;
        // the kernels index a mesh's work items in 32 bits
        for (int kind = 0; kind < W_COUNT; ++kind)
            if (items(kind, p->dim, (p->order - 1) / 2, nx[k], ny[k]) >= (1LL << 31)) return CGKS_EINVAL;
    }
    if ((r = load_tables())) return r;
    cgks_batch* b = new (std::nothrow) cgks_batch();
    if (!b) return CGKS_ENOMEM;
    b->p = *p;
    b->n = n;
    b->dim = p->dim;
    b->M = p->dim == 2 ? (p->order - 1) / 2 : 1;
    b->nvar = p->dim + 2;
    b->nplanes = p->dim == 2 ? 12 + 8 * b->M : 6;
    b->nacc = p->dim == 2 ? 4 + 8 * b->M : 6;
    b->rsize = p->precision == CGKS_FP64 ? 8 : 4;
    b->stream = (cudaStream_t)stream;
    if (!b->stream) {
        // graph capture needs a non-legacy stream: own one
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return CGKS_ECUDA; }
        b->own_stream = true;
    }
    b->k = pick_kfns(p->dim, p->order, p->precision, p->tau_mode, p->bc, p->pt_fallback, n == 1);
    std::vector<Layout> L(n);
    size_t total = 0;
    std::vector<size_t> base(n);
    for (int k = 0; k < n; ++k) {
        L[k] = layout(p->dim, b->M, b->rsize, nx[k], ny[k]);
        base[k] = total;
        total += L[k].total;
    }
    total = align256(total + n * sizeof(double));
    cudaError_t e = cudaMalloc(&b->slab, total);
    if (e != cudaSuccess) { delete b; return e == cudaErrorMemoryAllocation ? CGKS_ENOMEM : CGKS_ECUDA; }
    b->dfixed = (double*)(b->slab + total - align256(n * sizeof(double)));
    b->host.resize(n);
    double K = p->dim == 2 ? (4.0 - 2.0 * p->gamma) / (p->gamma - 1.0) : (3.0 - p->gamma) / (p->gamma - 1.0);
    for (int k = 0; k < n; ++k) {
        Mesh& g = b->host[k];
        std::memset(&g, 0, sizeof(g));
        g.nx = nx[k]; g.ny = ny[k]; g.order = p->order; g.oi = (p->order - 5) / 2;
        for (int s = 0; s < 4; ++s) g.bc[s] = p->bc[s];
        g.tau_mode = p->tau_mode;
        g.dff_lag = p->dff_lag;
        g.pf = p->pt_fallback;
        g.x0 = ext[4 * k];
        g.y0 = p->dim == 2 ? ext[4 * k + 2] : 0.0;
        std::memcpy(g.bcs, p->bc_state, sizeof(g.bcs));
        std::memcpy(g.bcx, p->bc_split, sizeof(g.bcx));
        g.dx = (ext[4 * k + 1] - ext[4 * k]) / nx[k];
        g.dy = p->dim == 2 ? (ext[4 * k + 3] - ext[4 * k + 2]) / ny[k] : 1.0;
        g.gamma = p->gamma; g.K = K; g.thr = p->sigma_thres; g.ghi = p->gamma_hi; g.glo = p->gamma_lo;
        g.eps = p->weno_eps; g.c1 = p->tau_c1; g.c2 = p->tau_c2; g.cfl = p->cfl;
        g.gf = (float)g.gamma; g.Kf = (float)g.K; g.c1f = (float)g.c1; g.c2f = (float)g.c2;
        g.idx = 1.0 / g.dx; g.idy = 1.0 / g.dy;
        g.mu = p->mu; g.muf = (float)p->mu;
        g.idxf = (float)g.idx; g.idyf = (float)g.idy;
        g.idxlo = (float)(g.idx - (double)g.idxf); g.idylo = (float)(g.idy - (double)g.idyf);
        g.plane = (long long)nx[k] * ny[k];
        char* m0 = b->slab + base[k];
        g.S0 = (double*)(m0 + L[k].S);
        g.S1 = g.S0 + (size_t)b->nplanes * g.plane;
        if (b->rsize == 4) {
            g.F0 = (float*)(m0 + L[k].F);
            g.F1 = g.F0 + (size_t)(b->nplanes + b->nvar) * g.plane;
        }
        g.ACC = (double*)(m0 + L[k].ACC);
        g.sig_x = (double*)(m0 + L[k].sigx);
        g.sig_xn = g.sig_x + (size_t)(nx[k] + 1) * ny[k];
        g.sig_y = p->dim == 2 ? (double*)(m0 + L[k].sigy) : nullptr;
        g.sig_yn = p->dim == 2 ? g.sig_y + (size_t)(ny[k] + 1) * nx[k] : nullptr;
        for (int d = 0; d < 2; ++d) {
            g.FR[d] = m0 + L[k].FR[d];
            g.FO[d] = m0 + L[k].FO[d];
            g.SP[d] = (double*)(m0 + L[k].SP[d]);
            g.AT[d] = m0 + L[k].AT[d];
            g.TD[d] = m0 + L[k].TD[d];
        }
        char* sc = m0 + L[k].scal;
        g.dt = (double*)sc;
        g.t = (double*)(sc + 8);
        g.status = (unsigned*)(sc + 16);
        g.bad = (long long*)(sc + 24);
        g.smax = (unsigned long long*)(sc + 32);
        g.branch = (unsigned long long*)(sc + 40);
        g.dtf = (float*)(sc + 72);
        g.ghost = (const double*)(sc + 80);  // 36 doubles of fixed ghost cells (1-D)
        g.tn = (double*)(sc + 368);
        g.nfall = (unsigned long long*)(sc + 376);
    }
    // prefix arrays
    b->off.assign((size_t)W_COUNT * (n + 1), 0);
    for (int kind = 0; kind < W_COUNT; ++kind)
        for (int k = 0; k < n; ++k)
            b->off[(size_t)kind * (n + 1) + k + 1] = b->off[(size_t)kind * (n + 1) + k] + items(kind, p->dim, b->M, nx[k], ny[k]);
    int rr = CGKS_OK;
    do {
        if (cudaMalloc(&b->dmesh, n * sizeof(Mesh)) != cudaSuccess) { rr = CGKS_ENOMEM; break; }
        if (cudaMalloc(&b->doff, b->off.size() * sizeof(long long)) != cudaSuccess) { rr = CGKS_ENOMEM; break; }
        if (cudaMemcpy(b->dmesh, b->host.data(), n * sizeof(Mesh), cudaMemcpyHostToDevice) != cudaSuccess) { rr = CGKS_ECUDA; break; }
        if (cudaMemcpy(b->doff, b->off.data(), b->off.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess) { rr = CGKS_ECUDA; break; }
        {
            std::vector<long long> one((size_t)n * W_COUNT * 2, 0);
            for (int k = 0; k < n; ++k)
                for (int kind = 0; kind < W_COUNT; ++kind)
                    one[((size_t)k * W_COUNT + kind) * 2 + 1] = items(kind, p->dim, b->M, nx[k], ny[k]);
            if (cudaMalloc(&b->doff1, one.size() * sizeof(long long)) != cudaSuccess) { rr = CGKS_ENOMEM; break; }
            if (cudaMemcpy(b->doff1, one.data(), one.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess) { rr = CGKS_ECUDA; break; }
        }
        // zero the scalars and scratch once (bad index = max)
        if (cudaMemsetAsync(b->slab, 0, total, b->stream) != cudaSuccess) { rr = CGKS_ECUDA; break; }
        for (int k = 0; k < n; ++k) {
            long long mx = LLONG_MAX;
            if (cudaMemcpyAsync(b->host[k].bad, &mx, 8, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) { rr = CGKS_ECUDA; break; }
        }
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) { rr = CGKS_ECUDA; break; }
        // persistent grids: SM count x resident blocks of each kernel
        int dev;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
        const void* fns[7] = {nullptr, (const void*)b->k.normal, (const void*)b->k.flux1,
                              (const void*)b->k.flux2, (const void*)b->k.upd1, (const void*)b->k.upd2,
                              (const void*)b->k.cfl};
        for (int q = 0; q < 7; ++q) {
            int occ = 1;
            int th = (q == 2 || q == 3) ? 128 : 256;
            b->threads[q] = th;
            if (fns[q]) {
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[q], th, 0) != cudaSuccess) occ = 1;
            }
            b->grid[q] = std::max(1, occ) * b->nsm;
        }
        // 2-D Steps 1-2: the default tile shape in both directions
        if (p->dim == 2)
            for (int d = 0; d < 2; ++d)
                if ((rr = set_tile(b, d, kTileShapes[0][0], kTileShapes[0][1], 256))) break;
    } while (0);
    if (rr) { cgks_batch_destroy(b); return rr; }
    *out = b;
    return CGKS_OK;
}

int status_of(cgks_batch* b, long long* bad_out)
{
    int rc = CGKS_OK;
    long long first = LLONG_MAX;
    for (int k = 0; k < b->n; ++k) {
        unsigned st = 0;
        long long bad = LLONG_MAX;
        CK(cudaMemcpy(&st, b->host[k].status, 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&bad, b->host[k].bad, 8, cudaMemcpyDeviceToHost));
        if (st & STATUS_NONPHYS) { rc = CGKS_ENONPHYS; first = std::min(first, bad); }
    }
    if (bad_out) *bad_out = rc ? first : -1;
    return rc;
}

int set_state_impl(cgks_batch* b, int k, const double* W, const double* Wx, const double* Wy,
                   const double* Wxl, const double* Wyl, const double* sx, const double* sy,
                   cudaMemcpyKind kind, bool sync)
{
    if (k < 0 || k >= b->n) return CGKS_EINVAL;
    Mesh& g = b->host[k];
    size_t P = (size_t)g.plane;
    int nv = b->nvar;
    if (!W || !Wx) return CGKS_EINVAL;
    if (b->dim == 2 && (!Wy || !Wxl || !Wyl)) return CGKS_EINVAL;
    cudaStream_t s = b->stream;
    CK(cudaMemcpyAsync(g.S0, W, nv * P * 8, kind, s));
    CK(cudaMemcpyAsync(g.S0 + nv * P, Wx, nv * P * 8, kind, s));
    if (b->dim == 2) {
        CK(cudaMemcpyAsync(g.S0 + 8 * P, Wy, 4 * P * 8, kind, s));
        CK(cudaMemcpyAsync(g.S0 + 12 * P, Wxl, 4 * b->M * P * 8, kind, s));
        CK(cudaMemcpyAsync(g.S0 + (12 + 4 * b->M) * P, Wyl, 4 * b->M * P * 8, kind, s));
    }
    CK(cudaMemsetAsync(g.status, 0, 4, s));
    CK(cudaMemsetAsync(g.t, 0, 8, s));
    CK(cudaMemsetAsync(g.tn, 0, 8, s));
    CK(cudaMemsetAsync(g.nfall, 0, 8, s));
    long long mx = LLONG_MAX;
    CK(cudaMemcpyAsync(g.bad, &mx, 8, cudaMemcpyHostToDevice, s));
    if (sx) {
        CK(cudaMemcpyAsync(g.sig_x, sx, (size_t)(g.nx + 1) * g.ny * 8, kind, s));
        if (b->dim == 2) {
            if (!sy) return CGKS_EINVAL;
            CK(cudaMemcpyAsync(g.sig_y, sy, (size_t)(g.ny + 1) * g.nx * 8, kind, s));
        }
    }
    if (sync) CK(cudaStreamSynchronize(s));
    return CGKS_OK;
}

// Run the per-mesh init kernels (sigma init when needed, positivity check)
// over the whole table after a set_state.
// Launch a per-mesh kernel over the items of mesh k alone.
int launch_one(cgks_batch* b, int k, const void* fn, int kind, int arg, bool has_arg)
{
    Work w;
    w.mesh = b->dmesh + k;
    w.m0 = b->host[k];
    w.off = b->doff1 + ((size_t)k * W_COUNT + kind) * 2;
    w.n = 1;
    w.total = items(kind, b->dim, b->M, b->host[k].nx, b->host[k].ny);
    if (w.total == 0) return CGKS_OK;
    int threads = 256;
    long long need = (w.total + threads - 1) / threads;
    int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)b->grid[6]));
    void* a2[] = {&w, &arg};
    void* a1[] = {&w};
    CK(cudaLaunchKernel(fn, dim3(grid), dim3(threads), has_arg ? a2 : a1, 0, b->stream));
    return CGKS_OK;
}

// After mesh k of a batch is set: its float planes, sigma and positivity check.
int post_set_one(cgks_batch* b, int k)
{
    int r;
    if (b->rsize == 4 && (r = launch_one(b, k, (const void*)b->k.convert, W_CELLS, 1, true))) return r;
    if ((r = launch_one(b, k, (const void*)b->k.siginit, W_SIGINIT, 0, false))) return r;
    if ((r = launch_one(b, k, (const void*)b->k.check, W_CELLS, 0, false))) return r;
    CK(cudaStreamSynchronize(b->stream));
    unsigned st = 0;
    CK(cudaMemcpy(&st, b->host[k].status, 4, cudaMemcpyDeviceToHost));
    return (st & STATUS_NONPHYS) ? CGKS_ENONPHYS : CGKS_OK;
}

// FP32-bulk form: the float planes follow the FP64 state after a set (to_float)
// and the FP64 slope planes follow the float planes before a read-out.
int convert_state(cgks_batch* b, int to_float)
{
    if (b->rsize != 4) return CGKS_OK;
    return launch(b, (const void*)b->k.convert, W_CELLS, 6, to_float, true);
}

int post_set(cgks_batch* b, bool init_sigma)
{
    int r;
    if ((r = convert_state(b, 1))) return r;
    if (init_sigma && (r = launch(b, (const void*)b->k.siginit, W_SIGINIT, 6, 0, false))) return r;
    if ((r = launch(b, (const void*)b->k.check, W_CELLS, 6, 0, false))) return r;
    CK(cudaStreamSynchronize(b->stream));
    return status_of(b, nullptr);
}

} // namespace

namespace {

// Persistent grid for a kernel at a given block size: SM count x resident blocks.
int grid_for(cgks_batch* b, const void* fn, int threads)
{
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0) != cudaSuccess || occ < 1) occ = 1;
    return occ * b->nsm;
}

// Time each stage kernel at every admissible block size on the current state
// and keep the fastest.  Only kernels that write scratch data run (stage 1
// lines / normal / flux / update and the stage-2 flux); the simulated time,
// the fallback count and the status word are restored afterwards.  The step
// graphs are rebuilt on next use.
int autotune(cgks_batch* b, int* out)
{
    if (!b->state_set) return CGKS_EINVAL;
    // tuning order: each kernel runs after the producers of its inputs (the
    // stage-2 flux last: it reads the stage-1 state W* that the update writes);
    // the 2-D Steps 1-2 are tuned first, over tile shapes and block sizes
    const void* fns[4] = {b->dim == 1 ? (const void*)b->k.normal : nullptr, (const void*)b->k.flux1,
                          (const void*)b->k.upd1, (const void*)b->k.flux2};
    const int slots[4] = {1, 2, 4, 3};
    const int kinds[4] = {W_NORMAL, W_FLUX, W_CELLS, W_FLUX};
    const int stages[4] = {1, 0, 0, 0};
    const bool has_stage[4] = {true, false, false, false};
    std::vector<double> t_saved(b->n), tn_saved(b->n);
    std::vector<unsigned long long> nf_saved(b->n);
    std::vector<unsigned> st_saved(b->n);
    std::vector<long long> bad_saved(b->n);
    for (int k = 0; k < b->n; ++k) {
        CK(cudaMemcpy(&t_saved[k], b->host[k].t, 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&tn_saved[k], b->host[k].tn, 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&nf_saved[k], b->host[k].nfall, 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&st_saved[k], b->host[k].status, 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&bad_saved[k], b->host[k].bad, 8, cudaMemcpyDeviceToHost));
    }
    // a CFL time step so that every kernel sees the data of a real step
    int r = launch(b, (const void*)b->k.cfl, W_CELLS, 6, 0, false);
    if (r) return r;
    {
        int use = 1;
        const double* fx = b->dfixed;
        Mesh* dm = b->dmesh;
        int nn = b->n;
        void* args[] = {&dm, &nn, &use, &fx};
        CK(cudaLaunchKernel((const void*)k_dt<0>, dim3((nn + 127) / 128), dim3(128), args, 0, b->stream));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int dir = 0; dir < (b->dim == 2 ? 2 : 0); ++dir) {
        float best = 1e30f;
        int bt = b->tile[dir][0], bb = b->tile[dir][1], bth = b->threads[dir];
        const int thr[2] = {128, 256};
        for (int sh = 0; sh < kNumTileShapes; ++sh)
            for (int c = 0; c < 2; ++c) {
                int TA = kTileShapes[sh][0], TB = kTileShapes[sh][1];
                if (set_tile(b, dir, TA, TB, thr[c]) != CGKS_OK) continue;  // no room on an SM
                float acc = 0.f;
                for (int rep = 0; rep < 4; ++rep) {
                    CK(cudaEventRecord(e0, b->stream));
                    if ((r = launch_recon(b, dir, 1))) return r;
                    CK(cudaEventRecord(e1, b->stream));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    if (rep > 0) acc += ms;  // the first launch warms caches
                }
                if (acc < best) { best = acc; bt = TA; bb = TB; bth = thr[c]; }
            }
        if ((r = set_tile(b, dir, bt, bb, bth))) return r;
    }
    for (int qq = 0; qq < 4; ++qq) {
        if (!fns[qq]) continue;
        int q = slots[qq];
        // the flux kernels come in two register variants; the others in one
        const void* var[2] = {fns[qq], nullptr};
        if (q == 2) { var[0] = (const void*)b->k.flux1v[0]; var[1] = (const void*)b->k.flux1v[1]; }
        if (q == 3) { var[0] = (const void*)b->k.flux2v[0]; var[1] = (const void*)b->k.flux2v[1]; }
        if (var[1] == var[0]) var[1] = nullptr;
        int best_t = b->threads[q], best_g = b->grid[q];
        const void* best_f = fns[qq];
        float best = 1e30f;
        const int cand[4] = {64, 128, 256, 512};
        for (int vi = 0; vi < 2; ++vi) {
            if (!var[vi]) continue;
            cudaFuncAttributes at;
            CK(cudaFuncGetAttributes(&at, var[vi]));
            for (int c = 0; c < 4; ++c) {
                int th = cand[c];
                if (th > at.maxThreadsPerBlock) continue;
                b->threads[q] = th;
                b->grid[q] = grid_for(b, var[vi], th);
                float acc = 0.f;
                for (int rep = 0; rep < 4; ++rep) {
                    CK(cudaEventRecord(e0, b->stream));
                    if ((r = launch(b, var[vi], kinds[qq], q, stages[qq], has_stage[qq]))) return r;
                    CK(cudaEventRecord(e1, b->stream));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    if (rep > 0) acc += ms;  // the first launch warms caches
                }
                if (acc < best) { best = acc; best_t = th; best_g = b->grid[q]; best_f = var[vi]; }
            }
        }
        b->threads[q] = best_t;
        b->grid[q] = best_g;
        if (q == 2) b->k.flux1 = (KOne)best_f;
        if (q == 3) b->k.flux2 = (KOne)best_f;
    }
    // stage-2 update shares the stage-1 update's shape
    b->threads[5] = b->threads[4];
    b->grid[5] = grid_for(b, (const void*)b->k.upd2, b->threads[5]);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int k = 0; k < b->n; ++k) {
        CK(cudaMemcpy(b->host[k].t, &t_saved[k], 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->host[k].tn, &tn_saved[k], 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->host[k].nfall, &nf_saved[k], 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->host[k].status, &st_saved[k], 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->host[k].bad, &bad_saved[k], 8, cudaMemcpyHostToDevice));
    }
    for (int g = 0; g < 2; ++g)
        if (b->gexec[g]) { cudaGraphExecDestroy(b->gexec[g]); b->gexec[g] = nullptr; }
    if (out) {
        for (int q = 0; q < 6; ++q) out[q] = b->threads[q];
        if (b->dim == 1) out[0] = 0;
        // register-capped flux variants are reported as a negative block size
        if (b->k.flux1v[1] != b->k.flux1v[0] && b->k.flux1 == b->k.flux1v[1]) out[2] = -out[2];
        if (b->k.flux2v[1] != b->k.flux2v[0] && b->k.flux2 == b->k.flux2v[1]) out[3] = -out[3];
        for (int d = 0; d < 2; ++d)
            for (int e = 0; e < 2; ++e) out[6 + 2 * d + e] = b->dim == 2 ? b->tile[d][e] : 0;
    }
    return CGKS_OK;
}

} // namespace

extern "C" {

int cgks_autotune(cgks_solver* s, int* threads_out)
{
    if (!s) return CGKS_EINVAL;
    return autotune(s->b, threads_out);
}

int cgks_batch_autotune(cgks_batch* b, int* threads_out)
{
    if (!b) return CGKS_EINVAL;
    return autotune(b, threads_out);
}

int cgks_default_params(cgks_params* p, int dim, int order)
{
    if (!p) return CGKS_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->dim = dim;
    p->order = order;
    p->precision = CGKS_FP64;
    p->tau_mode = CGKS_TAU_ZERO;
    p->gamma = 1.4;
    p->cfl = 0.5;
    p->sigma_thres = 1.0;
    p->gamma_hi = 0.85;
    p->gamma_lo = 0.6;
    p->weno_eps = 1e-8;
    p->tau_c1 = 0.05;
    p->tau_c2 = 1.0;
    p->dff_lag = CGKS_DFF_LAG_STEP;
    return CGKS_OK;
}

int cgks_init_mesh(cgks_solver** out, const cgks_params* p, int nx, int ny, double x0, double x1,
                   double y0, double y1, void* stream)
{
    if (!out) return CGKS_EINVAL;
    *out = nullptr;
    double ext[4] = {x0, x1, y0, y1};
    cgks_batch* b = nullptr;
    int r = batch_create(&b, p, 1, &nx, &ny, ext, stream);
    if (r) return r;
    cgks_solver* s = new (std::nothrow) cgks_solver();
    if (!s) { cgks_batch_destroy(b); return CGKS_ENOMEM; }
    s->b = b;
    *out = s;
    return CGKS_OK;
}

int cgks_set_state(cgks_solver* s, const double* W, const double* Wx, const double* Wy, const double* Wx_line,
                   const double* Wy_line, const double* sigma_x, const double* sigma_y)
{
    if (!s) return CGKS_EINVAL;
    int r = set_state_impl(s->b, 0, W, Wx, Wy, Wx_line, Wy_line, sigma_x, sigma_y, cudaMemcpyHostToDevice, true);
    if (r) return r;
    s->b->state_set = true;
    s->b->sigma_pending = sigma_x == nullptr;
    return post_set(s->b, sigma_x == nullptr);
}

int cgks_set_state_device(cgks_solver* s, const double* W, const double* Wx, const double* Wy,
                          const double* Wx_line, const double* Wy_line, const double* sigma_x,
                          const double* sigma_y)
{
    if (!s) return CGKS_EINVAL;
    int r = set_state_impl(s->b, 0, W, Wx, Wy, Wx_line, Wy_line, sigma_x, sigma_y, cudaMemcpyDeviceToDevice, false);
    if (r) return r;
    s->b->state_set = true;
    s->b->sigma_pending = sigma_x == nullptr;
    if ((r = convert_state(s->b, 1))) return r;
    if (sigma_x == nullptr) return launch(s->b, (const void*)s->b->k.siginit, W_SIGINIT, 6, 0, false);
    return CGKS_OK;
}

int cgks_set_ghost(cgks_solver* s, const double* ghost)
{
    if (!s || !ghost || s->b->dim != 1) return CGKS_EINVAL;
    CK(cudaMemcpy((void*)s->b->host[0].ghost, ghost, 36 * sizeof(double), cudaMemcpyHostToDevice));
    return CGKS_OK;
}

int cgks_set_time(cgks_solver* s, double t)
{
    if (!s || !std::isfinite(t)) return CGKS_EINVAL;
    cgks_batch* b = s->b;
    CK(cudaMemcpyAsync(b->host[0].t, &t, 8, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->host[0].tn, &t, 8, cudaMemcpyHostToDevice, b->stream));
    // a sigma that set_state initialised from the cell averages takes the
    // ghost states of inflow sides at this time, as if the state had been set at t
    if (b->sigma_pending) return launch(b, (const void*)b->k.siginit, W_SIGINIT, 6, 0, false);
    return CGKS_OK;
}

int cgks_compute_dt(cgks_solver* s, double* dt)
{
    if (!s || !dt) return CGKS_EINVAL;
    cgks_batch* b = s->b;
    int r = launch(b, (const void*)b->k.cfl, W_CELLS, 6, 0, false);
    if (r) return r;
    unsigned long long bits = 0, zero = 0;
    CK(cudaMemcpyAsync(&bits, b->host[0].smax, 8, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(b->host[0].smax, &zero, 8, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    double sm;
    std::memcpy(&sm, &bits, 8);
    *dt = sm > 0.0 ? b->p.cfl / sm : 0.0;
    return CGKS_OK;
}

int cgks_step(cgks_solver* s, double dt)
{
    if (!s) return CGKS_EINVAL;
    return cgks_advance(s, 1, dt);
}

int cgks_advance(cgks_solver* s, int n, double dt)
{
    if (!s || n < 0 || !s->b->state_set) return CGKS_EINVAL;
    cgks_batch* b = s->b;
    int which = dt > 0.0 ? 0 : 1;
    int r = build_graph(b, which);
    if (r) return r;
    if (n > 0) b->sigma_pending = false;
    for (int q = 0; q < n; ++q) {
        if (which == 0) {
            CK(cudaMemcpyAsync(b->dfixed, &dt, 8, cudaMemcpyHostToDevice, b->stream));
        }
        CK(cudaGraphLaunch(b->gexec[which], b->stream));
    }
    return CGKS_OK;
}

int cgks_sync(cgks_solver* s, double* t_out, long long* bad_cell)
{
    if (!s) return CGKS_EINVAL;
    CK(cudaStreamSynchronize(s->b->stream));
    if (t_out) CK(cudaMemcpy(t_out, s->b->host[0].t, 8, cudaMemcpyDeviceToHost));
    return status_of(s->b, bad_cell);
}

static int get_state_impl(cgks_batch* b, int k, double* W, double* Wx, double* Wy, double* Wxl, double* Wyl,
                          double* sx, double* sy, cudaMemcpyKind kind, bool sync)
{
    if (k < 0 || k >= b->n) return CGKS_EINVAL;
    Mesh& g = b->host[k];
    size_t P = (size_t)g.plane;
    int nv = b->nvar;
    cudaStream_t s = b->stream;
    if (b->state_set) {
        int r = convert_state(b, 0);
        if (r) return r;
    }
    if (W) CK(cudaMemcpyAsync(W, g.S0, nv * P * 8, kind, s));
    if (Wx) CK(cudaMemcpyAsync(Wx, g.S0 + nv * P, nv * P * 8, kind, s));
    if (b->dim == 2) {
        if (Wy) CK(cudaMemcpyAsync(Wy, g.S0 + 8 * P, 4 * P * 8, kind, s));
        if (Wxl) CK(cudaMemcpyAsync(Wxl, g.S0 + 12 * P, 4 * b->M * P * 8, kind, s));
        if (Wyl) CK(cudaMemcpyAsync(Wyl, g.S0 + (12 + 4 * b->M) * P, 4 * b->M * P * 8, kind, s));
        if (sy) CK(cudaMemcpyAsync(sy, g.sig_y, (size_t)(g.ny + 1) * g.nx * 8, kind, s));
    }
    if (sx) CK(cudaMemcpyAsync(sx, g.sig_x, (size_t)(g.nx + 1) * g.ny * 8, kind, s));
    if (sync) CK(cudaStreamSynchronize(s));
    return CGKS_OK;
}

int cgks_get_state(cgks_solver* s, double* W, double* Wx, double* Wy, double* Wx_line, double* Wy_line,
                   double* sigma_x, double* sigma_y)
{
    if (!s) return CGKS_EINVAL;
    return get_state_impl(s->b, 0, W, Wx, Wy, Wx_line, Wy_line, sigma_x, sigma_y, cudaMemcpyDeviceToHost, true);
}

int cgks_get_state_device(cgks_solver* s, double* W, double* Wx, double* Wy, double* Wx_line, double* Wy_line,
                          double* sigma_x, double* sigma_y)
{
    if (!s) return CGKS_EINVAL;
    return get_state_impl(s->b, 0, W, Wx, Wy, Wx_line, Wy_line, sigma_x, sigma_y, cudaMemcpyDeviceToDevice, false);
}

int cgks_get_stats(cgks_solver* s, cgks_stats* st)
{
    if (!s || !st) return CGKS_EINVAL;
    cgks_batch* b = s->b;
    Mesh& g = b->host[0];
    size_t P = (size_t)g.plane;
    int nv = b->nvar;
    std::vector<double> W(nv * P);
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaMemcpy(W.data(), g.S0, nv * P * 8, cudaMemcpyDeviceToHost));
    std::memset(st, 0, sizeof(*st));
    CK(cudaMemcpy(&st->t, g.t, 8, cudaMemcpyDeviceToHost));
    unsigned long long br[4];
    CK(cudaMemcpy(br, g.branch, sizeof(br), cudaMemcpyDeviceToHost));
    for (int q = 0; q < 4; ++q) st->branch[q] = (long long)br[q];
    unsigned long long nf = 0;
    CK(cudaMemcpy(&nf, g.nfall, 8, cudaMemcpyDeviceToHost));
    st->fallbacks = (long long)nf;
    st->min_rho = 1e300;
    st->min_p = 1e300;
    for (size_t c = 0; c < P; ++c) {
        double rho = W[c], u = W[P + c] / rho, v = b->dim == 2 ? W[2 * P + c] / rho : 0.0;
        double p = (b->p.gamma - 1.0) * (W[(b->dim + 1) * P + c] - 0.5 * rho * (u * u + v * v));
        st->min_rho = std::min(st->min_rho, rho);
        st->min_p = std::min(st->min_p, p);
        for (int q = 0; q < nv; ++q) st->mass[q] += W[q * P + c] * g.dx * g.dy;
    }
    return CGKS_OK;
}

int cgks_step_info(cgks_solver* s, int* kernels_per_step)
{
    if (!s || !kernels_per_step) return CGKS_EINVAL;
    int r = build_graph(s->b, 1);
    if (r) return r;
    *kernels_per_step = s->b->kernels_per_step;
    return CGKS_OK;
}

int cgks_profile_step(cgks_solver* s, double dt, float* ms, int* ids, int* n)
{
    if (!s || !ms || !ids || !n || *n < 1 || !(dt > 0.0) || !s->b->state_set) return CGKS_EINVAL;
    cgks_batch* b = s->b;
    cudaEvent_t ev[17];
    int cap = std::min(*n, 16), cnt = 0, r = CGKS_OK;
    for (int q = 0; q <= 16; ++q) CK(cudaEventCreate(&ev[q]));
    CK(cudaMemcpyAsync(b->dfixed, &dt, 8, cudaMemcpyHostToDevice, b->stream));
    CK(cudaEventRecord(ev[0], b->stream));
    auto rec = [&](int id) -> int {
        if (cnt < cap) {
            ids[cnt] = id;
            if (cudaEventRecord(ev[cnt + 1], b->stream) != cudaSuccess) return CGKS_ECUDA;
        }
        ++cnt;
        return CGKS_OK;
    };
    {
        int use = 0;
        const double* fx = b->dfixed;
        Mesh* dm = b->dmesh;
        int nn = b->n;
        void* args[] = {&dm, &nn, &use, &fx};
        CK(cudaLaunchKernel((const void*)k_dt<0>, dim3((nn + 127) / 128), dim3(128), args, 0, b->stream));
        if ((r = rec(4))) goto done;
    }
    for (int stage = 1; stage <= 2; ++stage) {
        if (b->dim == 2) {
            if ((r = launch_recon(b, 0, stage)) || (r = rec(10 * stage + 0))) goto done;
            if ((r = launch_recon(b, 1, stage)) || (r = rec(10 * stage + 1))) goto done;
        } else {
            if ((r = launch(b, (const void*)b->k.normal, W_NORMAL, 1, stage, true)) || (r = rec(10 * stage + 1))) goto done;
        }
        if ((r = launch(b, (const void*)(stage == 1 ? b->k.flux1 : b->k.flux2), W_FLUX, stage == 1 ? 2 : 3, 0, false)) ||
            (r = rec(10 * stage + 2))) goto done;
        if ((r = launch(b, (const void*)(stage == 1 ? b->k.upd1 : b->k.upd2), W_CELLS, stage == 1 ? 4 : 5, 0, false)) ||
            (r = rec(10 * stage + 3))) goto done;
    }
done:
    if (cudaStreamSynchronize(b->stream) != cudaSuccess && !r) r = CGKS_ECUDA;
    if (!r) {
        int m = std::min(cnt, cap);
        for (int q = 0; q < m; ++q)
            if (cudaEventElapsedTime(&ms[q], ev[q], ev[q + 1]) != cudaSuccess) r = CGKS_ECUDA;
        *n = m;
    }
    for (int q = 0; q <= 16; ++q) cudaEventDestroy(ev[q]);
    return r;
}

void cgks_destroy(cgks_solver* s)
{
    if (!s) return;
    cgks_batch_destroy(s->b);
    delete s;
}

const char* cgks_strerror(int code)
{
    switch (code) {
    case CGKS_OK: return "ok";
    case CGKS_EINVAL: return "invalid argument";
    case CGKS_ENOMEM: return "device allocation failed";
    case CGKS_ECUDA: return "CUDA runtime error";
    case CGKS_ENONPHYS: return "non-positive density or pressure, or non-finite value";
    case CGKS_ETIMEOUT: return "bounded device wait timed out";
    case CGKS_ENOTSUP: return "option combination not supported";
    default: return "unknown error";
    }
}

int cgks_batch_init(cgks_batch** out, const cgks_params* p, int n, const int* nx, const int* ny, const double* ext,
                    void* stream)
{
    if (p && p->dim != 2) return CGKS_EINVAL;
    return batch_create(out, p, n, nx, ny, ext, stream);
}

int cgks_batch_set_state(cgks_batch* b, int k, const double* W, const double* Wx, const double* Wy,
                         const double* Wx_line, const double* Wy_line)
{
    if (!b) return CGKS_EINVAL;
    int r = set_state_impl(b, k, W, Wx, Wy, Wx_line, Wy_line, nullptr, nullptr, cudaMemcpyHostToDevice, true);
    if (r) return r;
    b->state_set = true;
    return post_set_one(b, k);
}

int cgks_batch_set_state_device(cgks_batch* b, int k, const double* W, const double* Wx, const double* Wy,
                                const double* Wx_line, const double* Wy_line)
{
    if (!b) return CGKS_EINVAL;
    int r = set_state_impl(b, k, W, Wx, Wy, Wx_line, Wy_line, nullptr, nullptr, cudaMemcpyDeviceToDevice, false);
    if (r) return r;
    b->state_set = true;
    // the float planes, sigma from the cell averages and the positivity check of
    // instance k, enqueued; a non-physical state shows in cgks_batch_sync
    if (b->rsize == 4 && (r = launch_one(b, k, (const void*)b->k.convert, W_CELLS, 1, true))) return r;
    if ((r = launch_one(b, k, (const void*)b->k.siginit, W_SIGINIT, 0, false))) return r;
    return launch_one(b, k, (const void*)b->k.check, W_CELLS, 0, false);
}

int cgks_batch_get_state_device(cgks_batch* b, int k, double* W, double* Wx, double* Wy, double* Wx_line,
                                double* Wy_line)
{
    if (!b) return CGKS_EINVAL;
    return get_state_impl(b, k, W, Wx, Wy, Wx_line, Wy_line, nullptr, nullptr, cudaMemcpyDeviceToDevice, false);
}

int cgks_batch_step(cgks_batch* b, const double* dt)
{
    if (!b || !b->state_set) return CGKS_EINVAL;
    int which = dt ? 0 : 1;
    int r = build_graph(b, which);
    if (r) return r;
    if (dt) CK(cudaMemcpyAsync(b->dfixed, dt, b->n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    CK(cudaGraphLaunch(b->gexec[which], b->stream));
    return CGKS_OK;
}

int cgks_batch_sync(cgks_batch* b)
{
    if (!b) return CGKS_EINVAL;
    CK(cudaStreamSynchronize(b->stream));
    return status_of(b, nullptr);
}

int cgks_batch_get_state(cgks_batch* b, int k, double* W, double* Wx, double* Wy, double* Wx_line, double* Wy_line)
{
    if (!b) return CGKS_EINVAL;
    return get_state_impl(b, k, W, Wx, Wy, Wx_line, Wy_line, nullptr, nullptr, cudaMemcpyDeviceToHost, true);
}

void cgks_batch_destroy(cgks_batch* b)
{
    if (!b) return;
    for (int q = 0; q < 2; ++q)
        if (b->gexec[q]) cudaGraphExecDestroy(b->gexec[q]);
    if (b->dmesh) cudaFree(b->dmesh);
    if (b->doff) cudaFree(b->doff);
    if (b->doff1) cudaFree(b->doff1);
    if (b->slab) cudaFree(b->slab);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int cgks_stencil_row(int order, int st, int row, double* out)
{
    if (!out || st < 0 || st > 5 || row < 0 || row > 9) return CGKS_EINVAL;
    CgksTables t;
    if (cgks_build_tables(order, &t) != 0) return CGKS_EINVAL;
    if (row >= 6 + t.m) return CGKS_EINVAL;
    for (int k = 0; k < 10; ++k) out[k] = t.row[st][row][k];
    return CGKS_OK;
}

} // extern "C"

// ---------------------------------------------------------------- no-allocation 1-D step
//
// For callers that may not allocate device memory: every buffer a 1-D step
// needs besides the caller's state and sigma arrays lives in the file-scope
// array below.  The existing kernels run unchanged; only their descriptor
// points into this array.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CGKS_NOALLOC_SCRATCH_BYTES];

namespace {

const int kMaxDevices = 64;
unsigned char* g_noalloc_base[kMaxDevices];  // device address of the array, per device
std::mutex g_noalloc_mu;                     // host threads racing on a first call set up once

// Once per device, with that device current: the array's device address
// (host code must not use the array's name as an address) and the tables.
int noalloc_setup(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) return CGKS_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_base[dev]) return CGKS_OK;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return CGKS_ECUDA;
    int r = load_tables();
    if (r) return r;
    g_noalloc_base[dev] = (unsigned char*)ptr;
    return CGKS_OK;
}

// Everything a no-allocation step must place in the array before its stage
// kernels run, passed by value: kernel arguments are copied when the launch
// is enqueued, so no host memory is read later.
struct NoallocInit {
    Mesh g;
    long long off[W_COUNT * 2];
    double dt;  // > 0: the fixed step
};
static_assert(sizeof(NoallocInit) <= 4000, "kernel arguments are limited to 4 KB");

__global__ void k_noalloc_init(NoallocInit a, Mesh* dmesh, long long* doff, unsigned long long* scal)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int q = 0; q < 64; ++q) scal[q] = 0ull;  // the 512 bytes of scalars
    *dmesh = a.g;
    for (int q = 0; q < W_COUNT * 2; ++q) doff[q] = a.off[q];
    *a.g.bad = LLONG_MAX;
    if (a.dt > 0.0) *a.g.dt = a.dt;
}

} // namespace

extern "C" int cgks_step_1d_noalloc(const cgks_params* p, int nx, double x0, double x1,
                                    const double* state_in, const double* sigma_in,
                                    double* state_out, double* sigma_out, double dt,
                                    unsigned* status_out, void* stream)
{
    int r = validate(p);
    if (r) return r;
    if (p->dim != 1) return CGKS_EINVAL;
    if (p->bc[0] == CGKS_BC_FIXED || p->bc[1] == CGKS_BC_FIXED) return CGKS_ENOTSUP;
    if (nx < 1 || nx > CGKS_NOALLOC_MAX_CELLS || !(x1 > x0)) return CGKS_EINVAL;
    if ((p->bc[0] >= CGKS_BC_REFLECTIVE || p->bc[1] >= CGKS_BC_REFLECTIVE) && nx < 3) return CGKS_EINVAL;
    if (!state_in || !state_out || !sigma_out) return CGKS_EINVAL;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if ((r = noalloc_setup(dev))) return r;
    cudaStream_t st = (cudaStream_t)stream;
    size_t rs = p->precision == CGKS_FP64 ? 8 : 4;
    // carve the array: S1, ACC, sigma (new), FR, FO, SP, scalars, descriptor, offsets
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    size_t oS1 = take(6 * (size_t)nx * 8), oACC = take(6 * (size_t)nx * 8), oSN = take((size_t)(nx + 1) * 8);
    size_t oFR = take(3 * (size_t)(nx + 1) * 24 * rs), oFO = take((size_t)(nx + 1) * 16 * rs);
    size_t oSP = take((size_t)(nx + 1) * 8), oSC = take(512), oM = take(sizeof(Mesh));
    size_t oOF = take(W_COUNT * 2 * sizeof(long long));
    size_t oF = take(rs == 4 ? 2 * 9 * (size_t)nx * 4 : 0);  // FP32-bulk float planes and low parts
    if (o > CGKS_NOALLOC_SCRATCH_BYTES) return CGKS_EINVAL;
    unsigned char* base = g_noalloc_base[dev];
    Mesh g;
    std::memset(&g, 0, sizeof(g));
    g.nx = nx; g.ny = 1; g.order = p->order; g.oi = (p->order - 5) / 2;
    for (int q = 0; q < 4; ++q) g.bc[q] = p->bc[q];
    g.tau_mode = p->tau_mode;
    g.dff_lag = p->dff_lag;
    g.pf = p->pt_fallback;
    g.x0 = x0;
    g.dx = (x1 - x0) / nx; g.dy = 1.0;
    g.gamma = p->gamma; g.K = (3.0 - p->gamma) / (p->gamma - 1.0); g.thr = p->sigma_thres;
    g.ghi = p->gamma_hi; g.glo = p->gamma_lo; g.eps = p->weno_eps; g.c1 = p->tau_c1; g.c2 = p->tau_c2;
    g.cfl = p->cfl; g.plane = nx;
    g.gf = (float)g.gamma; g.Kf = (float)g.K; g.c1f = (float)g.c1; g.c2f = (float)g.c2;
    g.idx = 1.0 / g.dx; g.idy = 1.0;
    g.mu = p->mu; g.muf = (float)p->mu;
    g.idxf = (float)g.idx; g.idyf = 1.0f;
    g.idxlo = (float)(g.idx - (double)g.idxf); g.idylo = 0.0f;
    g.S0 = state_out;
    g.S1 = (double*)(base + oS1);
    if (rs == 4) {
        g.F0 = (float*)(base + oF);
        g.F1 = g.F0 + 9 * (size_t)nx;
    }
    g.ACC = (double*)(base + oACC);
    g.sig_x = sigma_out;
    g.sig_xn = (double*)(base + oSN);
    g.FR[0] = base + oFR; g.FO[0] = base + oFO; g.SP[0] = (double*)(base + oSP);
    unsigned char* sc = base + oSC;
    g.dt = (double*)sc; g.t = (double*)(sc + 8); g.status = (unsigned*)(sc + 16);
    g.bad = (long long*)(sc + 24); g.smax = (unsigned long long*)(sc + 32);
    g.branch = (unsigned long long*)(sc + 40); g.dtf = (float*)(sc + 72); g.ghost = (const double*)(sc + 80);
    g.tn = (double*)(sc + 368); g.nfall = (unsigned long long*)(sc + 376);
    NoallocInit init;
    std::memset(&init, 0, sizeof(init));
    init.g = g;
    const long long* off = init.off;
    for (int kind = 0; kind < W_COUNT; ++kind) { init.off[2 * kind] = 0; init.off[2 * kind + 1] = items(kind, 1, 1, nx, 1); }
    init.dt = dt;
    Mesh* dmesh = (Mesh*)(base + oM);
    long long* doff = (long long*)(base + oOF);
    // scalars start from zero (bad index from its maximum); descriptor, offsets
    // and the fixed step in, all as kernel arguments
    {
        unsigned long long* scal = (unsigned long long*)sc;
        void* args[] = {&init, &dmesh, &doff, &scal};
        CK(cudaLaunchKernel((const void*)k_noalloc_init, dim3(1), dim3(32), args, 0, st));
    }
    if (state_out != state_in) CK(cudaMemcpyAsync(state_out, state_in, 6 * (size_t)nx * 8, cudaMemcpyDeviceToDevice, st));
    if (sigma_in && sigma_in != sigma_out)
        CK(cudaMemcpyAsync(sigma_out, sigma_in, (size_t)(nx + 1) * 8, cudaMemcpyDeviceToDevice, st));
    Kfns k = pick_kfns(1, p->order, p->precision, p->tau_mode, p->bc, p->pt_fallback, true);
    int nsm = 1;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    auto go = [&](const void* fn, int kind, int stage, bool has_stage, int threads) -> int {
        Work w;
        w.mesh = dmesh;
        w.m0 = g;
        w.off = doff + 2 * kind;
        w.n = 1;
        w.total = off[2 * kind + 1];
        long long need = (w.total + threads - 1) / threads;
        int grid = (int)std::max<long long>(1, std::min<long long>(need, 4LL * nsm));
        void* a2[] = {&w, &stage};
        void* a1[] = {&w};
        CK(cudaLaunchKernel(fn, dim3(grid), dim3(threads), has_stage ? a2 : a1, 0, st));
        return CGKS_OK;
    };
    if (rs == 4 && (r = go((const void*)k.convert, W_CELLS, 1, true, 256))) return r;
    if (!sigma_in && (r = go((const void*)k.siginit, W_SIGINIT, 0, false, 256))) return r;
    // dt: the CFL reduction into the scratch scalars, or the fixed value copied above
    int use_cfl = dt > 0.0 ? 0 : 1;
    if (use_cfl && (r = go((const void*)k.cfl, W_CELLS, 0, false, 256))) return r;
    {
        int n1 = 1;
        const double* fixed = g.dt;
        void* args[] = {&dmesh, &n1, &use_cfl, &fixed};
        CK(cudaLaunchKernel((const void*)k_dt<0>, dim3(1), dim3(32), args, 0, st));
    }
    for (int stage = 1; stage <= 2; ++stage) {
        if ((r = go((const void*)k.normal, W_NORMAL, stage, true, 256))) return r;
        if ((r = go((const void*)(stage == 1 ? k.flux1 : k.flux2), W_FLUX, 0, false, 128))) return r;
        if ((r = go((const void*)(stage == 1 ? k.upd1 : k.upd2), W_CELLS, 0, false, 256))) return r;
    }
    if (rs == 4 && (r = go((const void*)k.convert, W_CELLS, 0, true, 256))) return r;
    if (status_out) CK(cudaMemcpyAsync(status_out, g.status, sizeof(unsigned), cudaMemcpyDeviceToDevice, st));
    return CGKS_OK;
}
