// Host-side pieces of restarted (F)GMRES shared by the single-system driver
// (htd_capi.cu) and the batch driver (htd_batch.cu): the Givens update of one
// Hessenberg column and the triangular solve for the update coefficients.
// Compiled without FMA contraction (build flag), so both drivers round alike.
#pragma once

#include <cmath>
#include <complex>

namespace htd {

typedef std::complex<double> zcd;

// Column j of the Hessenberg matrix (col[0..j+1], col[j+1] real >= 0): apply
// the rotations 0..j-1, then choose rotation j to zero col[j+1] and apply it
// to col and to the right-hand side g.
inline void givens_column(zcd *col, zcd *cs, double *sn, zcd *g, int j)
{
    for (int i = 0; i < j; ++i) {
        const zcd a = col[i], b = col[i + 1];
        col[i] = std::conj(cs[i]) * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    const zcd a = col[j];
    const double b = col[j + 1].real();
    const double rr = std::sqrt(std::norm(a) + b * b);
    if (rr == 0.0) {
        cs[j] = 1.0;
        sn[j] = 0.0;
    } else {
        cs[j] = a / rr;
        sn[j] = b / rr;
    }
    col[j] = std::conj(cs[j]) * a + sn[j] * b;
    col[j + 1] = 0.0;
    const zcd gj = g[j];
    g[j] = std::conj(cs[j]) * gj;
    g[j + 1] = -sn[j] * gj;
}

// y[0..jj) = R^{-1} g with R the leading jj x jj upper triangle of the rotated
// Hessenberg matrix stored by columns of length m + 1.
inline void solve_upper(const zcd *Hm, int m, const zcd *g, zcd *y, int jj)
{
    for (int i = jj - 1; i >= 0; --i) {
        zcd acc = g[i];
        for (int k = i + 1; k < jj; ++k) acc -= Hm[(size_t)k * (m + 1) + i] * y[k];
        y[i] = acc / Hm[(size_t)i * (m + 1) + i];
    }
}

}  // namespace htd
