// Reconstruction tables shared by the host generator and the CUDA kernels.
#pragma once

struct CgksTables {
    // stencil st (0 S0, 1 S1, 2 S2, 3 r5, 4 r7, 5 r9), functional row (see
    // tables.cpp), tap over [Qbar_{i-2..i+2}, h*Qx_{i-2..i+2}]
    double row[6][10][10];
    // polynomial coefficients c_0..c_4 of S0, S1, S2 (degree 2) and r5 (degree 4)
    double cpoly[4][5][10];
    // smoothness matrices (Eq. 3.13) of degree-2 and degree-4 polynomials
    double bm2[3][3];
    double bm4[5][5];
    // Gauss-Legendre nodes on [-1/2, 1/2] and weights summing to 1
    double gx[4], gw[4];
    // Step 3 first / second derivative weights over the 3m face points
    double d1[4][12], d2[4][12];
    int m;
};

#ifdef __cplusplus
extern "C"
#endif
__attribute__((visibility("hidden"))) int cgks_build_tables(int order, CgksTables* t);
