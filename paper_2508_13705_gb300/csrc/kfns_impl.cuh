// Instantiates the kernels of one configuration (included once per unit).
#pragma once
#include "cgks_kernels.cuh"
#include "kfns.h"

namespace cgks {
namespace {
int upload_tables(const CgksTables* t3, const TabF* f3)
{
    if (cudaMemcpyToSymbol(c_tab, t3, sizeof(CgksTables) * 3) != cudaSuccess) return 1;
    if (cudaMemcpyToSymbol(c_tabf, f3, sizeof(TabF) * 3) != cudaSuccess) return 1;
    return 0;
}
}  // namespace

template <int D, int M, typename R, bool ONE>
Kfns make_kfns_one()
{
    Kfns k;
    if constexpr (D == 2) {
        k.recon[0] = k_recon<M, R, false, 0, ONE>;
        k.recon[1] = k_recon<M, R, false, 1, ONE>;
        k.reconw[0] = k_recon<M, R, true, 0, ONE>;
        k.reconw[1] = k_recon<M, R, true, 1, ONE>;
        k.normal = k.normalw = nullptr;
    } else {
        k.recon[0] = k.recon[1] = k.reconw[0] = k.reconw[1] = nullptr;
        k.normal = k_normal1<R, false, ONE>;
        k.normalw = k_normal1<R, true, ONE>;
    }
    k.flux1v[0] = k_flux<D, M, R, 1, 0, 0, false, ONE>;
    k.flux2v[0] = k_flux<D, M, R, 2, 0, 0, false, ONE>;
    k.flux1h[0] = k_flux<D, M, R, 1, 0, 1, false, ONE>;
    k.flux2h[0] = k_flux<D, M, R, 2, 0, 1, false, ONE>;
    // the register-capped variants round exactly like the uncapped ones in
    // FP64 only (the compiler may contract the FP32 arithmetic differently),
    // so the FP32-bulk form offers the autotuner one variant
    if constexpr (sizeof(R) == 8) {
        k.flux1v[1] = k_flux<D, M, R, 1, 1, 0, false, ONE>;
        k.flux2v[1] = k_flux<D, M, R, 2, 1, 0, false, ONE>;
        k.flux1h[1] = k_flux<D, M, R, 1, 1, 1, false, ONE>;
        k.flux2h[1] = k_flux<D, M, R, 2, 1, 1, false, ONE>;
    } else {
        k.flux1v[1] = k.flux1v[0];
        k.flux2v[1] = k.flux2v[0];
        k.flux1h[1] = k.flux1h[0];
        k.flux2h[1] = k.flux2h[0];
    }
    k.flux1p = k_flux<D, M, R, 1, 0, 1, true, ONE>;
    k.flux2p = k_flux<D, M, R, 2, 0, 1, true, ONE>;
    k.flux1 = k.flux1v[0];
    k.flux2 = k.flux2v[0];
    if (D == 2) { k.upd1 = (KOne)k_update2<M, R, 1, ONE>; k.upd2 = (KOne)k_update2<M, R, 2, ONE>; }
    else { k.upd1 = (KOne)k_update1<R, 1, ONE>; k.upd2 = (KOne)k_update1<R, 2, ONE>; }
    k.cfl = k_cfl<D, R>;
    k.siginit = k_sigma_init<D>;
    k.check = k_check_state<D>;
    k.convert = k_convert<D, M>;
    k.upload = upload_tables;
    return k;
}

// The stage kernels for a launch over a single mesh (one = true: descriptor
// by value) or over a table of meshes.
template <int D, int M, typename R>
Kfns make_kfns(bool one)
{
    return one ? make_kfns_one<D, M, R, true>() : make_kfns_one<D, M, R, false>();
}
}  // namespace cgks
