// Kernel entry points of one (dimension, Gauss points, precision)
// configuration; each configuration is compiled in its own translation unit.
// one: the stage kernels for launches over a single mesh.
#pragma once
#include "cgks_device.cuh"

namespace cgks {
typedef void (*KStage)(Work, int);
typedef void (*KOne)(Work);
typedef void (*KTile)(Work, int, int, int);
struct Kfns {
    KTile recon[2];            // 2-D Steps 1-2 per direction (meshes without walls)
    KTile reconw[2];           // the same with the wall ghost rules
    KStage normal, normalw;    // 1-D Step 2, without and with the wall ghost rules
    KOne flux1, flux2, upd1, upd2, cfl, siginit, check;
    KStage convert;  // FP32-bulk state copies (to_float = 1: FP64 -> float planes)
    KOne flux1v[2], flux2v[2];  // flux variants: [0] uncapped, [1] register-capped (tau = 0)
    KOne flux1h[2], flux2h[2];  // the same with the collision-time terms (tau > 0)
    KOne flux1p, flux2p;        // tau > 0 with the first-order fallback at face points
    int (*upload)(const CgksTables* t3, const TabF* f3);  // constant tables of this unit
};
Kfns kfns_1_1_d(bool one);
Kfns kfns_1_1_f(bool one);
Kfns kfns_2_2_d(bool one);
Kfns kfns_2_3_d(bool one);
Kfns kfns_2_4_d(bool one);
Kfns kfns_2_2_f(bool one);
Kfns kfns_2_3_f(bool one);
Kfns kfns_2_4_f(bool one);
}
