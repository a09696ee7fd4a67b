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

template <int D, int M, typename R>
Kfns make_kfns()
{
    Kfns k;
    k.lines = D == 2 ? (KStage)k_lines<M, R, false> : nullptr;
    k.normal = k_normal<D, M, R, false>;
    k.linesw = D == 2 ? (KStage)k_lines<M, R, true> : nullptr;
    k.normalw = k_normal<D, M, R, true>;
    k.flux1v[0] = k_flux<D, M, R, 1, 0, 0>;
    k.flux2v[0] = k_flux<D, M, R, 2, 0, 0>;
    k.flux1v[1] = k_flux<D, M, R, 1, 1, 0>;
    k.flux2v[1] = k_flux<D, M, R, 2, 1, 0>;
    k.flux1h[0] = k_flux<D, M, R, 1, 0, 1>;
    k.flux2h[0] = k_flux<D, M, R, 2, 0, 1>;
    k.flux1h[1] = k_flux<D, M, R, 1, 1, 1>;
    k.flux2h[1] = k_flux<D, M, R, 2, 1, 1>;
    k.flux1p = k_flux<D, M, R, 1, 0, 1, true>;
    k.flux2p = k_flux<D, M, R, 2, 0, 1, true>;
    k.flux1 = k.flux1v[0];
    k.flux2 = k.flux2v[0];
    if (D == 2) { k.upd1 = (KOne)k_update2<M, R, 1>; k.upd2 = (KOne)k_update2<M, R, 2>; }
    else { k.upd1 = (KOne)k_update1<R, 1>; k.upd2 = (KOne)k_update1<R, 2>; }
    k.cfl = k_cfl<D, R>;
    k.siginit = k_sigma_init<D>;
    k.check = k_check_state<D>;
    k.convert = k_convert<D, M>;
    k.upload = upload_tables;
    return k;
}
}  // namespace cgks
