// Host-side generator of the reconstruction tables used by the CUDA kernels.
//
// Every Hermite stencil of Sec. 3.2 is a polynomial p(xi) on the unit local
// coordinate xi = (x - x_i)/h whose cell averages over [k-1/2, k+1/2] equal
// Qbar_{i+k} and whose slope averages p(k+1/2) - p(k-1/2) equal h*(Qx)_{i+k}
// on the cells the stencil draws from (Eq. 3.6-3.9, 3.18; the own-cell slope
// is not a condition).  The coefficients are obtained here by solving those
// conditions in extended precision (long double Gauss-Jordan) and are then
// turned into the linear functionals the kernels evaluate:
//   rows 0..2  value, d/dxi, d2/dxi2 at xi = +1/2  (left state of face i+1/2)
//   rows 3..5  the same at xi = -1/2               (right state of face i-1/2)
//   rows 6..   values at the Gauss nodes of the face (Step 1 line averages)
// plus the polynomial coefficients and smoothness-indicator matrices of the
// HWENO-AO(5,3) branch (Eq. 3.13), the Gauss-Legendre rule (Newton iteration
// on P_m) and the Step 3 derivative weights (least-squares polynomial of
// degree min(3m-1, 8) through the 3m face points of three segments).
#include <cmath>
#include <cstring>

#include "tables.h"

namespace {

typedef long double LD;

// Data layout of a stencil: [Qbar_{i-2..i+2}, h*Qx_{i-2..i+2}]
struct StencilDef { int navg; int avg[5]; int nslope; int slope[4]; };
const StencilDef kDefs[6] = {
    {2, {-1, 0}, 1, {-1}},                     // S0
    {2, {0, 1}, 1, {1}},                       // S1
    {3, {-1, 0, 1}, 0, {0}},                   // S2
    {3, {-1, 0, 1}, 2, {-1, 1}},               // r5
    {5, {-2, -1, 0, 1, 2}, 2, {-1, 1}},        // r7
    {5, {-2, -1, 0, 1, 2}, 4, {-2, -1, 1, 2}}, // r9
};

LD ipow(LD x, int n) { LD r = 1; for (int k = 0; k < n; ++k) r *= x; return r; }

// Solve A X = B in place (n x n, nrhs columns) by Gauss-Jordan with pivoting.
void gauss_jordan(LD* A, LD* B, int n, int nrhs)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
        if (p != c) {
            for (int t = 0; t < n; ++t) { LD x = A[c * n + t]; A[c * n + t] = A[p * n + t]; A[p * n + t] = x; }
            for (int t = 0; t < nrhs; ++t) { LD x = B[c * nrhs + t]; B[c * nrhs + t] = B[p * nrhs + t]; B[p * nrhs + t] = x; }
        }
        LD piv = A[c * n + c];
        for (int t = 0; t < n; ++t) A[c * n + t] /= piv;
        for (int t = 0; t < nrhs; ++t) B[c * nrhs + t] /= piv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            LD f = A[r * n + c];
            if (f == 0) continue;
            for (int t = 0; t < n; ++t) A[r * n + t] -= f * A[c * n + t];
            for (int t = 0; t < nrhs; ++t) B[r * nrhs + t] -= f * B[c * nrhs + t];
        }
    }
}

// coef[n][d]: polynomial coefficient n as a functional of the data entry d
void stencil_coefficients(int st, LD coef[9][10], int* deg_out)
{
    const StencilDef& S = kDefs[st];
    int n = S.navg + S.nslope;
    LD A[81], B[90];
    std::memset(B, 0, sizeof(B));
    int r = 0;
    for (int a = 0; a < S.navg; ++a, ++r) {
        LD lo = S.avg[a] - 0.5L, hi = S.avg[a] + 0.5L;
        for (int k = 0; k < n; ++k) A[r * n + k] = (ipow(hi, k + 1) - ipow(lo, k + 1)) / (k + 1);
        B[r * 10 + (S.avg[a] + 2)] = 1;
    }
    for (int a = 0; a < S.nslope; ++a, ++r) {
        LD lo = S.slope[a] - 0.5L, hi = S.slope[a] + 0.5L;
        for (int k = 0; k < n; ++k) A[r * n + k] = ipow(hi, k) - ipow(lo, k);
        B[r * 10 + 5 + (S.slope[a] + 2)] = 1;
    }
    gauss_jordan(A, B, n, 10);
    for (int k = 0; k < 9; ++k)
        for (int d = 0; d < 10; ++d) coef[k][d] = k < n ? B[k * 10 + d] : 0;
    *deg_out = n - 1;
}

// derivative nd of the polynomial at xi as a functional
void functional(LD coef[9][10], LD xi, int nd, double* out)
{
    for (int d = 0; d < 10; ++d) {
        LD s = 0;
        for (int k = nd; k < 9; ++k) {
            LD f = 1;
            for (int q = 0; q < nd; ++q) f *= (k - q);
            s += f * ipow(xi, k - nd) * coef[k][d];
        }
        out[d] = (double)s;
    }
}

// Gauss-Legendre rule on [-1/2, 1/2], weights summing to 1
void gauss_rule(int m, LD* x, LD* w)
{
    for (int i = 0; i < m; ++i) {
        LD z = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (m + 0.5L));
        for (int it = 0; it < 100; ++it) {
            LD p0 = 1, p1 = z;
            for (int k = 2; k <= m; ++k) { LD p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            LD dp = m * (z * p1 - p0) / (z * z - 1);
            LD dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-30L) break;
        }
        LD p0 = 1, p1 = z;
        for (int k = 2; k <= m; ++k) { LD p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
        LD dp = m * (z * p1 - p0) / (z * z - 1);
        x[m - 1 - i] = z / 2;
        w[m - 1 - i] = 1.0L / ((1 - z * z) * dp * dp); // 2/((1-z^2)P_m'(z)^2) on [-1,1], normalised to sum 1
    }
}

// least-squares polynomial of degree deg through (nodes, values): weights of
// its first and second derivatives at x
void lsq_derivative_weights(const LD* nodes, int n, int deg, LD x, double* d1, double* d2)
{
    int q = deg + 1;
    LD A[144], B[144];
    for (int a = 0; a < q; ++a) {
        for (int b = 0; b < q; ++b) {
            LD s = 0;
            for (int k = 0; k < n; ++k) s += ipow(nodes[k], a) * ipow(nodes[k], b);
            A[a * q + b] = s;
        }
        for (int k = 0; k < n; ++k) B[a * n + k] = ipow(nodes[k], a);
    }
    gauss_jordan(A, B, q, n);
    for (int k = 0; k < n; ++k) {
        LD s1 = 0, s2 = 0;
        for (int a = 1; a < q; ++a) s1 += B[a * n + k] * a * ipow(x, a - 1);
        for (int a = 2; a < q; ++a) s2 += B[a * n + k] * a * (a - 1) * ipow(x, a - 2);
        d1[k] = (double)s1;
        d2[k] = (double)s2;
    }
}

// smoothness matrix of Eq. 3.13 for polynomials of degree deg over the
// coefficients c_1..c_deg: beta = sum_{a,b} c_a c_b M[a][b]
void smoothness_matrix(int deg, double* M /* (deg+1)^2 */)
{
    int n = deg + 1;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            LD s = 0;
            for (int q = 1; q <= deg; ++q) {
                if (a < q || b < q) continue;
                LD fa = 1, fb = 1;
                for (int r = 0; r < q; ++r) { fa *= (a - r); fb *= (b - r); }
                int e = a - q + b - q;
                if (e % 2) continue;
                s += fa * fb * 2 * ipow(0.5L, e + 1) / (e + 1);
            }
            M[a * n + b] = (double)s;
        }
}

} // namespace

extern "C" __attribute__((visibility("hidden"))) int cgks_build_tables(int order, CgksTables* t)
{
    if (!t || (order != 5 && order != 7 && order != 9)) return -1;
    std::memset(t, 0, sizeof(*t));
    int m = (order - 1) / 2;
    t->m = m;
    LD gx[4], gw[4];
    gauss_rule(m, gx, gw);
    for (int l = 0; l < m; ++l) { t->gx[l] = (double)gx[l]; t->gw[l] = (double)gw[l]; }
    for (int st = 0; st < 6; ++st) {
        LD coef[9][10];
        int deg;
        stencil_coefficients(st, coef, &deg);
        for (int s = 0; s < 2; ++s)
            for (int nd = 0; nd < 3; ++nd)
                functional(coef, s == 0 ? 0.5L : -0.5L, nd, t->row[st][s * 3 + nd]);
        for (int l = 0; l < m; ++l) functional(coef, gx[l], 0, t->row[st][6 + l]);
        if (st <= 3)
            for (int k = 0; k < 5; ++k)
                for (int d = 0; d < 10; ++d) t->cpoly[st][k][d] = (double)coef[k][d];
    }
    smoothness_matrix(2, &t->bm2[0][0]);
    smoothness_matrix(4, &t->bm4[0][0]);
    // Step 3: 3m nodes of segments b-1, b, b+1 (in units of the tangential h)
    LD nodes[12];
    for (int s = 0; s < 3; ++s)
        for (int l = 0; l < m; ++l) nodes[s * m + l] = (s - 1) + gx[l];
    int deg = 3 * m - 1 < 8 ? 3 * m - 1 : 8;
    for (int l = 0; l < m; ++l) lsq_derivative_weights(nodes, 3 * m, deg, gx[l], t->d1[l], t->d2[l]);
    return 0;
}
