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

// Classical Gram-Schmidt with one re-orthogonalisation (CGS2).  The new vector
// w is built in basis slot k, so one dot kernel over slots 0..k gives both
// V_i^H w (i < k) and ||w||^2 (slot k); each pass then subtracts w -= V h.
// With h0 (pass 1) and h1 (pass 2) the k + 1 results of the two passes, the
// Hessenberg column is h0 + h1 and the norm after pass 2 is
// ||w_1||^2 - |h1|^2 (Pythagoras; h1 is small against w_1, so no cancellation),
// which saves a third pass over w for its norm.
template <typename C2>
inline double cgs2_column(const C2 *h0, const C2 *h1, int k, zcd *col)
{
    double hh = 0.0;
    for (int i = 0; i < k; ++i) {
        col[i] = zcd(h0[i].x + h1[i].x, h0[i].y + h1[i].y);
        hh += h1[i].x * h1[i].x + h1[i].y * h1[i].y;
    }
    return h1[k].x - hh;
}

// Selective re-orthogonalisation ("twice is enough": Daniel, Gragg, Kaufman
// and Stewart 1976; Giraud, Langou and Rozloznik 2005).  After pass 1 (h0,
// k + 1 results) the new vector's squared norm is ||w_1||^2 = ||w||^2 - |h0|^2
// (Pythagoras against the orthonormal V).  If ||w_1||^2 >= ||w||^2 / 2 the
// projection lost at most one bit and one pass keeps w_1 orthogonal to V to
// working precision: the column is h0 and ||w_1||^2 is returned through *w1sq
// (no cancellation: the subtracted part is at most half).  Otherwise (or if a
// value is not finite) a second pass is needed and cgs2_column completes it.
template <typename C2>
inline bool cgs_needs_second_pass(const C2 *h0, int k, double *w1sq)
{
    double hh = 0.0;
    for (int i = 0; i < k; ++i) hh += h0[i].x * h0[i].x + h0[i].y * h0[i].y;
    const double w2 = h0[k].x;
    *w1sq = w2 - hh;
    return !(*w1sq >= 0.5 * w2);
}

template <typename C2>
inline void cgs1_column(const C2 *h0, int k, zcd *col)
{
    for (int i = 0; i < k; ++i) col[i] = zcd(h0[i].x, h0[i].y);
}

}  // namespace htd
