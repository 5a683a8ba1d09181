// Dense generalized symmetric-definite eigensolver for the small augmented
// problem F_A U = lambda F_B U (Sec. 3.3), host side.
//
// Reduction to standard form with the Cholesky factor of F_B, Householder
// tridiagonalisation, the k smallest eigenvalues by bisection on Sturm
// sequence counts, eigenvectors of the tridiagonal matrix by inverse
// iteration (with re-orthogonalisation inside clusters of close
// eigenvalues), then back-transformation.  The O(m^3) loops are split over
// OpenMP threads.
//
// Published methods used here: Householder tridiagonalisation; all the
// eigenvalues of a symmetric tridiagonal matrix by the implicit-shift QL
// iteration of Bowdler, Martin, Reinsch and Wilkinson (Numer. Math. 11,
// 1968; Wilkinson shift, deflation on negligible off-diagonal entries),
// `tridiag_eigvals`; Sturm-sequence bisection and inverse iteration
// (Wilkinson, The Algebraic Eigenvalue Problem, 1965).
#include "small_eig.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

namespace nas {

// sum_k a[k] b[k] with four interleaved partial sums (k mod 4), added as
// ((s0 + s1) + (s2 + s3)) + tail: a fixed order, and the four running sums
// let consecutive multiply-adds overlap instead of waiting on one sum
static inline double dot(const double* a, const double* b, int n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 4 <= n; k += 4) {
        s0 += a[k] * b[k];
        s1 += a[k + 1] * b[k + 1];
        s2 += a[k + 2] * b[k + 2];
        s3 += a[k + 3] * b[k + 3];
    }
    double s = (s0 + s1) + (s2 + s3);
    for (; k < n; ++k) s += a[k] * b[k];
    return s;
}

// Matrices of at least kParMin rows run their O(m^3) loops on all OpenMP
// threads (below that the fork/join cost exceeds the work).
static const int kParMin = 128;

// lower Cholesky in place (row-major, lower triangle); returns false if not SPD
static bool cholesky(int m, std::vector<double>& L) {
    for (int j = 0; j < m; ++j) {
        const double* Lj = &L[(size_t)j * m];
        double d = L[(size_t)j * m + j] - dot(Lj, Lj, j);
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        L[(size_t)j * m + j] = d;
#pragma omp parallel for schedule(static) if (m - j > 256 || (m >= kParMin && m - j > 64))
        for (int i = j + 1; i < m; ++i) {
            double* Li = &L[(size_t)i * m];
            Li[j] = (Li[j] - dot(Li, Lj, j)) / d;
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j) L[(size_t)i * m + j] = 0.0;
    return true;
}

// C = L^{-1} A L^{-T} (A symmetric, full storage built from its lower triangle)
// by two forward eliminations Z <- L^{-1} Z on all m columns at once, first
// of A, then of the transpose of the result.  Each elimination is
// left-looking over blocks of 8 columns: row i of the block is
// (B_i - sum_{k<i} L_ik Z_k) / L_ii with the 8 partial sums in registers and
// k ascending, so each L_ik is loaded once per 8 updates and each Z_k block
// once per row; the column blocks are independent and split over the OpenMP
// threads.
static void solve_lower_rows(int m, const std::vector<double>& L, std::vector<double>& Z) {
    const int kCb = 8;
    const int nblk = (m + kCb - 1) / kCb;
#pragma omp parallel for schedule(static) if (m >= kParMin)
    for (int b = 0; b < nblk; ++b) {
        const int j0 = b * kCb, w = std::min(kCb, m - j0);
        for (int i = 0; i < m; ++i) {
            const double* Li = &L[(size_t)i * m];
            double acc[kCb];
            double* zi = &Z[(size_t)i * m + j0];
            for (int q = 0; q < kCb; ++q) acc[q] = q < w ? zi[q] : 0.0;
            if (w == kCb) {
                for (int k = 0; k < i; ++k) {
                    const double l = Li[k];
                    const double* zk = &Z[(size_t)k * m + j0];
#pragma omp simd
                    for (int q = 0; q < kCb; ++q) acc[q] -= l * zk[q];
                }
            } else {
                for (int k = 0; k < i; ++k) {
                    const double l = Li[k];
                    const double* zk = &Z[(size_t)k * m + j0];
                    for (int q = 0; q < w; ++q) acc[q] -= l * zk[q];
                }
            }
            const double d = Li[i];
            for (int q = 0; q < w; ++q) zi[q] = acc[q] / d;
        }
    }
}

static void reduce_standard(int m, const std::vector<double>& L, const double* A, std::vector<double>& C) {
    std::vector<double> Y((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j <= i; ++j) Y[(size_t)i * m + j] = Y[(size_t)j * m + i] = A[(size_t)i * m + j];
    solve_lower_rows(m, L, Y);           // Y = L^-1 A
    C.resize((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) C[(size_t)i * m + j] = Y[(size_t)j * m + i];
    solve_lower_rows(m, L, C);           // C = L^-1 (L^-1 A)^T = L^-1 A L^-T
    // symmetrise
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < i; ++j) {
            double v = 0.5 * (C[(size_t)i * m + j] + C[(size_t)j * m + i]);
            C[(size_t)i * m + j] = v;
            C[(size_t)j * m + i] = v;
        }
}

// Householder tridiagonalisation of symmetric C (row-major; only the lower
// triangle is read and updated).  Reflector j acts on entries j+1..m-1:
// H_j = I - tau_j v_j v_j^T with v_j stored in V (row j), v_j[j+1] = 1.
// T = Q^T C Q, Q = H_0 H_1 ... H_{m-3}.
static void tridiagonalise_par(int m, std::vector<double>& C, std::vector<double>& d, std::vector<double>& e,
                               std::vector<double>& V, std::vector<double>& tau);

static void tridiagonalise(int m, std::vector<double>& C, std::vector<double>& d, std::vector<double>& e,
                           std::vector<double>& V, std::vector<double>& tau) {
    if (m >= kParMin) {
        tridiagonalise_par(m, C, d, e, V, tau);
        return;
    }
    d.assign(m, 0.0);
    e.assign(std::max(m - 1, 0), 0.0);
    V.assign((size_t)m * m, 0.0);
    tau.assign(m, 0.0);
    std::vector<double> p(m), w(m), v(m);
    for (int j = 0; j + 2 < m; ++j) {
        int n1 = m - j - 1;  // length of x = C[j+1:, j]
        double* x = &v[0];
        double xnorm2 = 0.0;
        for (int i = 0; i < n1; ++i) {
            x[i] = C[(size_t)(j + 1 + i) * m + j];
            if (i > 0) xnorm2 += x[i] * x[i];
        }
        double alpha = x[0];
        if (xnorm2 == 0.0) {
            tau[j] = 0.0;
            e[j] = alpha;
            continue;
        }
        double beta = -std::copysign(std::sqrt(alpha * alpha + xnorm2), alpha);
        double t = (beta - alpha) / beta;
        double scale = 1.0 / (alpha - beta);
        for (int i = 1; i < n1; ++i) x[i] *= scale;
        x[0] = 1.0;
        tau[j] = t;
        e[j] = beta;
        for (int i = 0; i < n1; ++i) V[(size_t)j * m + j + 1 + i] = x[i];
        // p = tau * C22 v from the lower triangle: row i contributes its dot
        // with v to p_i and, through the mirrored entries, v_i times the row
        // to p_0..p_{i-1}
        for (int i = 0; i < n1; ++i) p[i] = 0.0;
        for (int i = 0; i < n1; ++i) {
            const double* Ci = &C[(size_t)(j + 1 + i) * m + j + 1];
            const double xi = x[i];
            double s0 = 0.0, s1 = 0.0;
            int k = 0;
            for (; k + 2 <= i; k += 2) {
                s0 += Ci[k] * x[k];
                s1 += Ci[k + 1] * x[k + 1];
                p[k] += Ci[k] * xi;
                p[k + 1] += Ci[k + 1] * xi;
            }
            for (; k < i; ++k) {
                s0 += Ci[k] * x[k];
                p[k] += Ci[k] * xi;
            }
            p[i] += (s0 + s1) + Ci[i] * xi;
        }
        for (int i = 0; i < n1; ++i) p[i] *= t;
        double pv = 0.0;
        for (int i = 0; i < n1; ++i) pv += p[i] * x[i];
        for (int i = 0; i < n1; ++i) w[i] = p[i] - 0.5 * t * pv * x[i];
        // C22 -= v w^T + w v^T (lower triangle)
        for (int i = 0; i < n1; ++i) {
            double* Ci = &C[(size_t)(j + 1 + i) * m + j + 1];
            const double xi = x[i], wi = w[i];
            for (int k = 0; k <= i; ++k) Ci[k] -= xi * w[k] + wi * x[k];
        }
    }
    for (int i = 0; i < m; ++i) d[i] = C[(size_t)i * m + i];
    if (m >= 2) e[m - 2] = C[(size_t)(m - 1) * m + (m - 2)];
}

// The same reflectors on all threads: C is mirrored to full storage, so the
// product p = tau C22 v and the update C22 -= v w^T + w v^T are row-parallel
// over whole rows (twice the multiply-adds of the lower-triangle form, no
// write conflicts); one parallel region for all steps, barriers between the
// phases of a step.
static void tridiagonalise_par(int m, std::vector<double>& C, std::vector<double>& d, std::vector<double>& e,
                               std::vector<double>& V, std::vector<double>& tau) {
    d.assign(m, 0.0);
    e.assign(std::max(m - 1, 0), 0.0);
    V.assign((size_t)m * m, 0.0);
    tau.assign(m, 0.0);
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < i; ++k) C[(size_t)k * m + i] = C[(size_t)i * m + k];
    std::vector<double> p(m), w(m), v(m);
    double t = 0.0, pv = 0.0;
    bool skip = false;
#pragma omp parallel
    for (int j = 0; j + 2 < m; ++j) {
        const int n1 = m - j - 1;
#pragma omp single
        {
            double* x = v.data();
            double xnorm2 = 0.0;
            for (int i = 0; i < n1; ++i) {
                x[i] = C[(size_t)(j + 1 + i) * m + j];
                if (i > 0) xnorm2 += x[i] * x[i];
            }
            const double alpha = x[0];
            skip = (xnorm2 == 0.0);
            if (skip) {
                tau[j] = 0.0;
                e[j] = alpha;
            } else {
                const double beta = -std::copysign(std::sqrt(alpha * alpha + xnorm2), alpha);
                t = (beta - alpha) / beta;
                const double scale = 1.0 / (alpha - beta);
                for (int i = 1; i < n1; ++i) x[i] *= scale;
                x[0] = 1.0;
                tau[j] = t;
                e[j] = beta;
                for (int i = 0; i < n1; ++i) V[(size_t)j * m + j + 1 + i] = x[i];
            }
        }  // implicit barrier
        if (skip) continue;  // every thread sees the same flag after the barrier
#pragma omp for schedule(static)
        for (int i = 0; i < n1; ++i) p[i] = t * dot(&C[(size_t)(j + 1 + i) * m + j + 1], v.data(), n1);
#pragma omp single
        {
            pv = dot(p.data(), v.data(), n1);
            for (int i = 0; i < n1; ++i) w[i] = p[i] - 0.5 * t * pv * v[i];
        }
#pragma omp for schedule(static)
        for (int i = 0; i < n1; ++i) {
            double* Ci = &C[(size_t)(j + 1 + i) * m + j + 1];
            const double xi = v[i], wi = w[i];
            for (int k = 0; k < n1; ++k) Ci[k] -= xi * w[k] + wi * v[k];
        }
    }
    for (int i = 0; i < m; ++i) d[i] = C[(size_t)i * m + i];
    if (m >= 2) e[m - 2] = C[(size_t)(m - 1) * m + (m - 2)];
}

// number of eigenvalues of T smaller than x (Sturm count of the LDL^T pivots)
static int sturm_count(int m, const std::vector<double>& d, const std::vector<double>& e, double x) {
    const double tiny = std::numeric_limits<double>::min();
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < m; ++i) {
        if (std::fabs(q) < tiny) q = -tiny;
        q = (d[i] - x) - e[i - 1] * e[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// LU factorisation with partial pivoting of (T - lam I), T tridiagonal, for
// repeated solves (inverse iteration).  U has diagonal 1/ainv, super-diagonal
// c and second super-diagonal u2; row i+1 was swapped with row i when
// swp[i], and l[i] is the multiplier of the elimination step i.
struct TriWork {
    std::vector<double> ainv, c, u2, l;
    std::vector<char> swp;
};

static void tri_factor(int m, const std::vector<double>& d, const std::vector<double>& e, double lam,
                       double pert, TriWork& w) {
    w.ainv.resize(m);
    w.c.resize(m);
    w.u2.assign(m, 0.0);
    w.l.assign(m, 0.0);
    w.swp.assign(m, 0);
    double* a = w.ainv.data();
    double* c = w.c.data();
    double* u2 = w.u2.data();
    for (int i = 0; i < m; ++i) {
        a[i] = d[i] - lam;
        c[i] = (i + 1 < m) ? e[i] : 0.0;
    }
    for (int i = 0; i + 1 < m; ++i) {
        const double sub = e[i];  // entry (i+1, i)
        if (std::fabs(a[i]) >= std::fabs(sub)) {
            if (a[i] == 0.0) a[i] = pert;
            const double l = sub / a[i];
            a[i + 1] -= l * c[i];
            w.l[i] = l;
        } else {
            // swap rows i and i+1
            const double l = a[i] / sub;
            const double ai1 = a[i + 1], ci1 = (i + 1 < m - 1) ? c[i + 1] : 0.0;
            a[i] = sub;
            const double ci = c[i];
            c[i] = ai1;
            u2[i] = ci1;
            a[i + 1] = ci - l * ai1;
            if (i + 1 < m - 1) c[i + 1] = -l * ci1;
            w.l[i] = l;
            w.swp[i] = 1;
        }
    }
    if (a[m - 1] == 0.0) a[m - 1] = pert;
    for (int i = 0; i < m; ++i) a[i] = 1.0 / a[i];
}

// b <- (T - lam I)^-1 b with the factors of tri_factor
static void tri_apply(int m, const TriWork& w, double* b) {
    const double* a = w.ainv.data();
    const double* c = w.c.data();
    const double* u2 = w.u2.data();
    for (int i = 0; i + 1 < m; ++i) {
        if (w.swp[i]) std::swap(b[i], b[i + 1]);
        b[i + 1] -= w.l[i] * b[i];
    }
    b[m - 1] *= a[m - 1];
    if (m >= 2) b[m - 2] = (b[m - 2] - c[m - 2] * b[m - 1]) * a[m - 2];
    for (int i = m - 3; i >= 0; --i) b[i] = (b[i] - c[i] * b[i + 1] - u2[i] * b[i + 2]) * a[i];
}

// sqrt(f^2 + g^2), with the scaled library routine only outside the range
// where the squares can neither overflow nor underflow
static inline double fast_hypot(double f, double g) {
    const double a = std::fmax(std::fabs(f), std::fabs(g));
    if (a > 1e-140 && a < 1e140) return std::sqrt(f * f + g * g);
    return std::hypot(f, g);
}

static bool tridiag_eigvals(int m, const std::vector<double>& d_in, const std::vector<double>& e_in,
                            std::vector<double>& w) {
    std::vector<double> d(d_in.begin(), d_in.begin() + m), e(m, 0.0);
    for (int i = 0; i + 1 < m; ++i) e[i] = e_in[i];
    const double eps = std::numeric_limits<double>::epsilon();
    for (int l = 0; l < m; ++l) {
        for (int sweep = 0;; ++sweep) {
            // end of the unreduced block that starts at l
            int mm = l;
            while (mm + 1 < m && std::fabs(e[mm]) > eps * (std::fabs(d[mm]) + std::fabs(d[mm + 1]))) ++mm;
            if (mm == l) break;
            if (sweep >= 60) return false;
            // shift: eigenvalue of the leading 2 x 2 corner closer to d[l]
            const double theta = (d[l + 1] - d[l]) / (2.0 * e[l]);
            const double rho = fast_hypot(theta, 1.0);
            const double shift = d[l] - e[l] / (theta + std::copysign(rho, theta));
            // implicit shifted QL step on rows l..mm, bottom to top
            double g = d[mm] - shift;
            double c = 1.0, sn = 1.0, p = 0.0;
            bool split = false;
            for (int i = mm - 1; i >= l; --i) {
                const double f = sn * e[i], b = c * e[i];
                const double r = fast_hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {  // the block splits at i+1: undo the pending shift there
                    d[i + 1] -= p;
                    e[mm] = 0.0;
                    split = true;
                    break;
                }
                sn = f / r;
                c = g / r;
                const double h = d[i + 1] - p;
                const double t = (d[i] - h) * sn + 2.0 * c * b;
                p = sn * t;
                d[i + 1] = h + p;
                g = c * t - b;
            }
            if (split) continue;
            d[l] -= p;
            e[l] = g;
            e[mm] = 0.0;
        }
    }
    std::sort(d.begin(), d.end());
    w.swap(d);
    return true;
}

// dense_gen_eig with the Cholesky factor L of B given (row-major lower)
static void gen_eig_factored(int m, const double* A, const std::vector<double>& L, int k, double* lam, double* U) {
    std::vector<double> C;
    reduce_standard(m, L, A, C);
    std::vector<double> d, e, V, tau;
    tridiagonalise(m, C, d, e, V, tau);
    // Gershgorin interval
    double lo = 1e300, hi = -1e300, tnorm = 0.0;
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
        tnorm = std::max(tnorm, std::fabs(d[i]) + r);
    }
    const double eps = std::numeric_limits<double>::epsilon();
    lo -= 2 * eps * tnorm + 1e-300;
    hi += 2 * eps * tnorm + 1e-300;
    std::vector<double> w(k);
    // many eigenvalues of a small matrix: QL (no serial chain of divisions per
    // bisection step); a few of a large one: bisection on the Sturm count
    bool have_w = false;
    if (m <= 512 && 4 * k >= m) {
        std::vector<double> all;
        if (tridiag_eigvals(m, d, e, all)) {
            for (int i = 0; i < k; ++i) w[i] = all[i];
            have_w = true;
        }
    }
#pragma omp parallel for schedule(dynamic, 1) if (!have_w)
    for (int i = 0; i < (have_w ? 0 : k); ++i) {
        double a = lo, b = hi;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (a + b);
            if (mid <= a || mid >= b) break;
            if (sturm_count(m, d, e, mid) > i)
                b = mid;
            else
                a = mid;
            if (b - a <= 2.0 * eps * std::max(std::fabs(a), std::fabs(b)) + 1e-300) break;
        }
        w[i] = 0.5 * (a + b);
    }
    // eigenvectors of T by inverse iteration; clusters re-orthogonalised
    std::vector<double> Z((size_t)k * m);
    const double pert = eps * tnorm + 1e-300;
    const double clus = 1e-3 * tnorm;
    // clusters of close eigenvalues [cstart[c], cstart[c+1]): vectors of one
    // cluster are orthogonalised against each other in order; different
    // clusters are independent
    std::vector<int> cstart{0};
    for (int i = 1; i < k; ++i)
        if (std::fabs(w[i] - w[i - 1]) > clus) cstart.push_back(i);
    cstart.push_back(k);
    const int ncl = (int)cstart.size() - 1;
#pragma omp parallel for schedule(dynamic, 1) if (m >= kParMin)
    for (int cl = 0; cl < ncl; ++cl) {
        std::vector<double> x(m);
        TriWork tw;
        const int start = cstart[cl];
        for (int i = start; i < cstart[cl + 1]; ++i) {
            for (int r = 0; r < m; ++r) x[r] = 1.0 + 0.01 * std::sin(0.7 * r + 1.3 * i);
            tri_factor(m, d, e, w[i], pert, tw);
            for (int it = 0; it < 4; ++it) {
                tri_apply(m, tw, x.data());
                for (int j = start; j < i; ++j) {
                    const double* zj = &Z[(size_t)j * m];
                    const double s = dot(zj, x.data(), m);
                    for (int r = 0; r < m; ++r) x[r] -= s * zj[r];
                }
                double nrm = std::sqrt(dot(x.data(), x.data(), m));
                if (!(nrm > 0)) {
                    for (int r = 0; r < m; ++r) x[r] = (r == i) ? 1.0 : 0.0;
                    nrm = 1.0;
                }
                for (int r = 0; r < m; ++r) x[r] /= nrm;
            }
            std::copy(x.begin(), x.end(), Z.begin() + (size_t)i * m);
        }
    }
    // back-transform: y = Q z = H_0 ... H_{m-3} z, then U = L^{-T} y (rows of
    // L^T, i.e. columns of L, made contiguous first)
    std::vector<double> Lt((size_t)m * m);
    for (int r = 0; r < m; ++r)
        for (int q = 0; q <= r; ++q) Lt[(size_t)q * m + r] = L[(size_t)r * m + q];
#pragma omp parallel for schedule(dynamic, 1) if (m >= kParMin || (int64_t)k * m * m > 2000000)
    for (int i = 0; i < k; ++i) {
        double* z = &Z[(size_t)i * m];
        for (int j = m - 3; j >= 0; --j) {
            if (tau[j] == 0.0) continue;
            const double* v = &V[(size_t)j * m];
            const double s = tau[j] * dot(v + j + 1, z + j + 1, m - j - 1);
            for (int r = j + 1; r < m; ++r) z[r] -= s * v[r];
        }
        // solve L^T u = z (backward)
        for (int r = m - 1; r >= 0; --r)
            z[r] = (z[r] - dot(&Lt[(size_t)r * m + r + 1], z + r + 1, m - r - 1)) / Lt[(size_t)r * m + r];
    }
    // Rayleigh quotients refine the eigenvalues: lambda = u^T A u (u is
    // B-normalised), from the lower triangle of A: sum_r u_r (A_rr u_r + 2 sum_{c<r} A_rc u_c)
#pragma omp parallel for schedule(dynamic, 1) if (m >= kParMin || (int64_t)k * m * m > 2000000)
    for (int i = 0; i < k; ++i) {
        const double* u = &Z[(size_t)i * m];
        double s = 0.0;
        for (int r = 0; r < m; ++r) {
            const double* Ar = A + (size_t)r * m;
            s += u[r] * (Ar[r] * u[r] + 2.0 * dot(Ar, u, r));
        }
        lam[i] = s;
    }
    for (int r = 0; r < m; ++r)
        for (int i = 0; i < k; ++i) U[(size_t)r * k + i] = Z[(size_t)i * m + r];
}

int dense_gen_eig(int m, const double* A, const double* B, int k, double* lam, double* U) {
    if (k > m) return -1;
    std::vector<double> L((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j <= i; ++j) L[(size_t)i * m + j] = B[(size_t)i * m + j];
    if (!cholesky(m, L)) return -1;
    gen_eig_factored(m, A, L, k, lam, U);
    return 0;
}

int chol_factor(int m, double* A) {
    std::vector<double> L(A, A + (size_t)m * m);
    if (!cholesky(m, L)) return -1;
    std::copy(L.begin(), L.end(), A);
    return 0;
}

void chol_inverse(int m, const double* L, double* Inv) {
    // U = L^T row-major, so that the backward solve reads contiguous rows
    std::vector<double> U((size_t)m * m);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int j = 0; j <= i; ++j) U[(size_t)j * m + i] = L[(size_t)i * m + j];
#pragma omp parallel
    {
        std::vector<double> y(m);
#pragma omp for schedule(dynamic, 8)
        for (int c = 0; c < m; ++c) {
            // L y = e_c: y vanishes above row c
            std::fill(y.begin(), y.end(), 0.0);
            y[c] = 1.0 / L[(size_t)c * m + c];
            for (int i = c + 1; i < m; ++i) {
                const double* Li = L + (size_t)i * m;
                double s = 0.0;
                for (int j = c; j < i; ++j) s -= Li[j] * y[j];
                y[i] = s / Li[i];
            }
            // L^T x = y
            for (int i = m - 1; i >= 0; --i) {
                const double* Ui = &U[(size_t)i * m];
                double s = y[i];
                for (int j = i + 1; j < m; ++j) s -= Ui[j] * y[j];
                y[i] = s / Ui[i];
            }
            // column c of the (symmetric) inverse, stored as row c
            std::copy(y.begin(), y.end(), Inv + (size_t)c * m);
        }
    }
}

void chol_solve(int m, const double* L, int k, double* B) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < k; ++c) {
        std::vector<double> y(m);
        for (int i = 0; i < m; ++i) {
            double s = B[(size_t)i * k + c];
            const double* Li = L + (size_t)i * m;
            for (int j = 0; j < i; ++j) s -= Li[j] * y[j];
            y[i] = s / Li[i];
        }
        for (int i = m - 1; i >= 0; --i) {
            double s = y[i];
            for (int j = i + 1; j < m; ++j) s -= L[(size_t)j * m + i] * y[j];
            y[i] = s / L[(size_t)i * m + i];
        }
        for (int i = 0; i < m; ++i) B[(size_t)i * k + c] = y[i];
    }
}

void jacobi_eig(int m, double* A, double* w, double* V) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) V[i * m + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                tot += A[i * m + j] * A[i * m + j];
                if (i != j) off += A[i * m + j] * A[i * m + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                double apq = A[p * m + q];
                if (apq == 0.0) continue;
                if (std::fabs(apq) <= 1e-18 * std::sqrt(std::fabs(A[p * m + p] * A[q * m + q]))) {
                    A[p * m + q] = A[q * m + p] = 0.0;
                    continue;
                }
                double theta = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                double t = std::copysign(1.0, theta) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {
                    double akp = A[k * m + p], akq = A[k * m + q];
                    A[k * m + p] = c * akp - s * akq;
                    A[k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {
                    double apk = A[p * m + k], aqk = A[q * m + k];
                    A[p * m + k] = c * apk - s * aqk;
                    A[q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    double vkp = V[k * m + p], vkq = V[k * m + q];
                    V[k * m + p] = c * vkp - s * vkq;
                    V[k * m + q] = s * vkp + c * vkq;
                }
            }
    }
    // sort ascending
    std::vector<int> idx(m);
    for (int i = 0; i < m; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[a * m + a] < A[b * m + b]; });
    std::vector<double> Vs(m * m);
    for (int j = 0; j < m; ++j) {
        w[j] = A[idx[j] * m + idx[j]];
        for (int i = 0; i < m; ++i) Vs[i * m + j] = V[i * m + idx[j]];
    }
    std::memcpy(V, Vs.data(), sizeof(double) * m * m);
}

int small_solve(int n, const double* A, const double* b, double* x) {
    if (n < 0 || n > 16) return -1;
    double M[16][17];
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) M[i][j] = A[i * n + j];
        M[i][n] = b[i];
    }
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[r][c]) > std::fabs(M[p][c])) p = r;
        if (M[p][c] == 0.0) return -1;
        if (p != c)
            for (int j = 0; j <= n; ++j) std::swap(M[p][j], M[c][j]);
        for (int r = c + 1; r < n; ++r) {
            double l = M[r][c] / M[c][c];
            for (int j = c; j <= n; ++j) M[r][j] -= l * M[c][j];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = M[i][n];
        for (int j = i + 1; j < n; ++j) s -= M[i][j] * x[j];
        x[i] = s / M[i][i];
    }
    return 0;
}

}  // namespace nas

// ------------------------------------------------------------------ LOBPCG
namespace nas {

// Y[m][k] = F X[m][k]
static void arrow_apply(const ArrowMat& F, int k, const double* X, double* Y) {
    const int64_t nH = F.nH;
    const int Na = F.Na;
    const int64_t m = nH + Na;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nH; ++i) {
        double* y = Y + i * k;
        for (int j = 0; j < k; ++j) y[j] = 0.0;
        for (int p = F.ptr[i]; p < F.ptr[i + 1]; ++p) {
            const double v = F.sval[p];
            const double* x = X + (int64_t)F.col[p] * k;
            for (int j = 0; j < k; ++j) y[j] += v * x[j];
        }
        for (int a = 0; a < Na; ++a) {
            const double v = F.Bd[i * Na + a];
            const double* x = X + (nH + a) * k;
            for (int j = 0; j < k; ++j) y[j] += v * x[j];
        }
    }
    // border rows: Bd^T X_H + Cd X_a (reduction over nH, split by columns)
#pragma omp parallel for schedule(static)
    for (int a = 0; a < Na; ++a) {
        double* y = Y + (nH + a) * k;
        for (int j = 0; j < k; ++j) y[j] = 0.0;
        for (int64_t i = 0; i < nH; ++i) {
            const double v = F.Bd[i * Na + a];
            const double* x = X + i * k;
            for (int j = 0; j < k; ++j) y[j] += v * x[j];
        }
        for (int b = 0; b < Na; ++b) {
            const double v = F.Cd[a * Na + b];
            const double* x = X + (nH + b) * k;
            for (int j = 0; j < k; ++j) y[j] += v * x[j];
        }
    }
    (void)m;
}

static double arrow_diag(const ArrowMat& F, int64_t i) {
    if (i < F.nH) {
        for (int p = F.ptr[i]; p < F.ptr[i + 1]; ++p)
            if (F.col[p] == i) return F.sval[p];
        return 0.0;
    }
    int64_t a = i - F.nH;
    return F.Cd[a * F.Na + a];
}

// G[ns][ns] = S^T T (S, T are [m][ns] row-major).  Rows are split into a
// fixed number of chunks; each chunk accumulates its outer products S_i^T T_i
// (contiguous rows), and the chunk sums are added in chunk order, so the
// result does not depend on the thread count.
static void gram(int64_t m, int ns, const double* S, const double* T, double* G) {
    const int chunks = 32;
    std::vector<double> part((size_t)chunks * ns * ns, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int ch = 0; ch < chunks; ++ch) {
        double* acc = &part[(size_t)ch * ns * ns];
        const int64_t i0 = m * ch / chunks, i1 = m * (ch + 1) / chunks;
        for (int64_t i = i0; i < i1; ++i) {
            const double* si = S + i * ns;
            const double* ti = T + i * ns;
            for (int a = 0; a < ns; ++a) {
                const double sa = si[a];
                if (sa == 0.0) continue;
                double* row = acc + (size_t)a * ns;
                for (int b = 0; b < ns; ++b) row[b] += sa * ti[b];
            }
        }
    }
    for (int q = 0; q < ns * ns; ++q) {
        double v = 0.0;
        for (int ch = 0; ch < chunks; ++ch) v += part[(size_t)ch * ns * ns + q];
        G[q] = v;
    }
}

// Y[m][kout] = S[m][ns] C[ns][kout]
static void mult(int64_t m, int ns, const double* S, int kout, const double* Cm, double* Y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double* y = Y + i * kout;
        for (int j = 0; j < kout; ++j) y[j] = 0.0;
        for (int a = 0; a < ns; ++a) {
            const double s = S[i * ns + a];
            if (s == 0.0) continue;
            const double* c = Cm + a * kout;
            for (int j = 0; j < kout; ++j) y[j] += s * c[j];
        }
    }
}

// All eigenpairs of a small symmetric matrix (ascending): the tridiagonal
// solver with B = I.  A is not modified; V [m][m] row-major, columns = vectors.
static void sym_eig_all(int m, const double* A, double* w, double* V) {
    std::vector<double> I((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) I[(size_t)i * m + i] = 1.0;
    if (dense_gen_eig(m, A, I.data(), m, w, V) != 0) {
        std::vector<double> Ac(A, A + (size_t)m * m);
        jacobi_eig(m, Ac.data(), w, V);
    }
}

// Rayleigh-Ritz on basis S [m][ns] with AS, BS: lowest k Ritz pairs.  The basis
// Gram matrix G = S^T B S is diagonalised; directions with eigenvalue below
// 1e-9 * max are dropped.  Returns coefficient matrix Y [ns][k] and theta[k].
static int rayleigh_ritz(int64_t m, int ns, const double* S, const double* AS, const double* BS, int k,
                         std::vector<double>& Y, std::vector<double>& theta) {
    std::vector<double> G((size_t)ns * ns), H((size_t)ns * ns);
    gram(m, ns, S, BS, G.data());
    gram(m, ns, S, AS, H.data());
    return rayleigh_ritz_grams(ns, G, H, k, Y, theta);
}

int rayleigh_ritz_grams(int ns, std::vector<double>& G, std::vector<double>& H, int k, std::vector<double>& Y,
                        std::vector<double>& theta, bool* fallback) {
    if (fallback) *fallback = false;
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < a; ++b) {
            double g = 0.5 * (G[a * ns + b] + G[b * ns + a]);
            G[a * ns + b] = G[b * ns + a] = g;
            double h = 0.5 * (H[a * ns + b] + H[b * ns + a]);
            H[a * ns + b] = H[b * ns + a] = h;
        }
    // fast path: a well-conditioned basis Gram matrix is factored by Cholesky
    // and the pencil (H, G) solved directly; the smallest squared pivot must
    // stay above 1e-8 of the largest diagonal entry (kappa(G) below ~1e8, so
    // the B-orthonormality of S Y holds to ~1e-12).  Otherwise the two-pass
    // eigen-decomposition below drops the near-dependent directions.
    {
        double gmax = 0.0;
        for (int a = 0; a < ns; ++a) gmax = std::max(gmax, G[(size_t)a * ns + a]);
        std::vector<double> L(G);
        if (gmax > 0.0 && cholesky(ns, L)) {
            double pmin = 1e300;
            for (int a = 0; a < ns; ++a) pmin = std::min(pmin, L[(size_t)a * ns + a] * L[(size_t)a * ns + a]);
            if (pmin >= 1e-8 * gmax) {
                std::vector<double> lam(k), U((size_t)ns * k);
                gen_eig_factored(ns, H.data(), L, k, lam.data(), U.data());
                theta.assign(lam.begin(), lam.end());
                Y.swap(U);
                return 0;
            }
        }
    }
    if (fallback) *fallback = true;
    // the O(ns^3) products below split their output rows over the OpenMP
    // threads; every entry keeps its summation order
    const bool par = ns >= kParMin;
    std::vector<double> gw(ns), GV((size_t)ns * ns);
    sym_eig_all(ns, G.data(), gw.data(), GV.data());
    double gmax = gw[ns - 1];
    // directions with Gram eigenvalue below 1e-9 * max are dropped: the Gram
    // matrix is only known to ~eps * max in absolute terms
    std::vector<int> keep;
    for (int a = 0; a < ns; ++a)
        if (gw[a] > 1e-9 * gmax) keep.push_back(a);
    int r = (int)keep.size();
    if (r < k) return -1;
    // Q = V_keep D^-1/2  [ns][r]
    std::vector<double> Q((size_t)ns * r);
    for (int a = 0; a < ns; ++a)
        for (int j = 0; j < r; ++j) Q[a * r + j] = GV[a * ns + keep[j]] / std::sqrt(gw[keep[j]]);
    // second pass: Q <- Q V2 D2^-1/2 with Q^T G Q = V2 D2 V2^T (restores B-orthonormality)
    {
        std::vector<double> GQ((size_t)ns * r), G2((size_t)r * r), w2(r), V2((size_t)r * r);
#pragma omp parallel for schedule(static) if (par)
        for (int a = 0; a < ns; ++a)
            for (int j = 0; j < r; ++j) {
                double sacc = 0.0;
                for (int b = 0; b < ns; ++b) sacc += G[a * ns + b] * Q[b * r + j];
                GQ[a * r + j] = sacc;
            }
#pragma omp parallel for schedule(static) if (par)
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < r; ++j) {
                double sacc = 0.0;
                for (int a = 0; a < ns; ++a) sacc += Q[a * r + i] * GQ[a * r + j];
                G2[i * r + j] = sacc;
            }
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < i; ++j) G2[i * r + j] = G2[j * r + i] = 0.5 * (G2[i * r + j] + G2[j * r + i]);
        sym_eig_all(r, G2.data(), w2.data(), V2.data());
        std::vector<double> Q2((size_t)ns * r);
#pragma omp parallel for schedule(static) if (par)
        for (int a = 0; a < ns; ++a)
            for (int j = 0; j < r; ++j) {
                double sacc = 0.0;
                for (int i = 0; i < r; ++i) sacc += Q[a * r + i] * V2[i * r + j];
                Q2[a * r + j] = sacc / std::sqrt(w2[j]);
            }
        Q.swap(Q2);
    }
    // Hr = Q^T H Q
    std::vector<double> HQ((size_t)ns * r), Hr((size_t)r * r);
#pragma omp parallel for schedule(static) if (par)
    for (int a = 0; a < ns; ++a)
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int b = 0; b < ns; ++b) s += H[a * ns + b] * Q[b * r + j];
            HQ[a * r + j] = s;
        }
#pragma omp parallel for schedule(static) if (par)
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int a = 0; a < ns; ++a) s += Q[a * r + i] * HQ[a * r + j];
            Hr[i * r + j] = s;
        }
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < i; ++j) Hr[i * r + j] = Hr[j * r + i] = 0.5 * (Hr[i * r + j] + Hr[j * r + i]);
    std::vector<double> hw(r), HV((size_t)r * r);
    sym_eig_all(r, Hr.data(), hw.data(), HV.data());
    theta.assign(hw.begin(), hw.begin() + k);
    Y.assign((size_t)ns * k, 0.0);
#pragma omp parallel for schedule(static) if (par)
    for (int a = 0; a < ns; ++a)
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int i = 0; i < r; ++i) s += Q[a * r + i] * HV[i * r + j];
            Y[a * k + j] = s;
        }
    return 0;
}

int lobpcg_arrow(const ArrowMat& A, const ArrowMat& B, int nev, int nguard, double* lam, double* U, bool warm,
                 double tol, int maxit) {
    const int64_t m = A.nH + A.Na;
    const int k = (int)std::min<int64_t>(nev + nguard, m);
    if (nev > m) return -1;
    std::vector<double> X((size_t)m * k), AX((size_t)m * k), BX((size_t)m * k);
    // start: warm vectors for the wanted columns, deterministic pseudo-random otherwise
    for (int64_t i = 0; i < m; ++i)
        for (int j = 0; j < k; ++j) {
            double r = std::sin(12.9898 * (i + 1) + 78.233 * (j + 1)) * 43758.5453;
            X[i * k + j] = r - std::floor(r) - 0.5;
        }
    if (warm)
        for (int64_t i = 0; i < m; ++i)
            for (int j = 0; j < nev; ++j) X[i * k + j] = U[i * nev + j];
    std::vector<double> dA(m), dB(m), T(m);
    for (int64_t i = 0; i < m; ++i) {
        dA[i] = arrow_diag(A, i);
        dB[i] = arrow_diag(B, i);
    }
    std::vector<double> Y, theta;
    auto refresh = [&]() {
        arrow_apply(A, k, X.data(), AX.data());
        arrow_apply(B, k, X.data(), BX.data());
    };
    refresh();
    if (rayleigh_ritz(m, k, X.data(), AX.data(), BX.data(), k, Y, theta) != 0) return -1;
    {
        std::vector<double> t((size_t)m * k);
        mult(m, k, X.data(), k, Y.data(), t.data());
        X.swap(t);
        refresh();
    }
    // diagonal preconditioner diag(A - sigma B)^-1 with sigma below the spectrum
    double sigma = theta[0] - 0.1 * std::fabs(theta[0]) - 1.0;
    for (int64_t i = 0; i < m; ++i) {
        double d = dA[i] - sigma * dB[i];
        T[i] = d > 0 ? 1.0 / d : 1.0;
    }
    std::vector<double> P, AP, BP;  // previous search directions [m][np]
    int np = 0;
    int it = 0;
    std::vector<double> rel(k);
    for (; it < maxit; ++it) {
        std::vector<double> rn(k, 0.0), an(k, 0.0), bn(k, 0.0);
#pragma omp parallel for schedule(static)
        for (int j = 0; j < k; ++j) {
            double r2 = 0.0, a2 = 0.0, b2 = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                double r = AX[i * k + j] - theta[j] * BX[i * k + j];
                r2 += r * r;
                a2 += AX[i * k + j] * AX[i * k + j];
                b2 += BX[i * k + j] * BX[i * k + j];
            }
            rn[j] = r2;
            an[j] = a2;
            bn[j] = b2;
        }
        double worst = 0.0;
        for (int j = 0; j < k; ++j) {
            rel[j] = std::sqrt(rn[j]) / (std::sqrt(an[j]) + std::fabs(theta[j]) * std::sqrt(bn[j]) + 1e-300);
            if (j < nev) worst = std::max(worst, rel[j]);
        }
        if (worst <= tol) break;
        // active columns: unconverged wanted vectors and every guard vector (soft locking)
        std::vector<int> act;
        for (int j = 0; j < k; ++j)
            if (j >= nev || rel[j] > 0.1 * tol) act.push_back(j);
        const int ka = (int)act.size();
        std::vector<double> W((size_t)m * ka);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i)
            for (int q = 0; q < ka; ++q) {
                int j = act[q];
                W[i * ka + q] = T[i] * (AX[i * k + j] - theta[j] * BX[i * k + j]);
            }
        // W <- W - X (BX)^T W, then unit B-norm columns (keeps the Gram matrix well scaled)
        {
            std::vector<double> Cm((size_t)k * ka), XC((size_t)m * ka);
            {
                const int chunks = 32;
                std::vector<double> part((size_t)chunks * k * ka, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
                for (int ch = 0; ch < chunks; ++ch) {
                    double* acc = &part[(size_t)ch * k * ka];
                    const int64_t i0 = m * ch / chunks, i1 = m * (ch + 1) / chunks;
                    for (int64_t i = i0; i < i1; ++i)
                        for (int a = 0; a < k; ++a) {
                            const double v = BX[i * k + a];
                            for (int b = 0; b < ka; ++b) acc[a * ka + b] += v * W[i * ka + b];
                        }
                }
                for (int q = 0; q < k * ka; ++q) {
                    double v = 0.0;
                    for (int ch = 0; ch < chunks; ++ch) v += part[(size_t)ch * k * ka + q];
                    Cm[q] = v;
                }
            }
            mult(m, k, X.data(), ka, Cm.data(), XC.data());
            for (size_t q = 0; q < W.size(); ++q) W[q] -= XC[q];
        }
        std::vector<double> AW((size_t)m * ka), BW((size_t)m * ka);
        arrow_apply(B, ka, W.data(), BW.data());
        {
            std::vector<double> nrm(ka, 0.0);
            for (int64_t i = 0; i < m; ++i)
                for (int q = 0; q < ka; ++q) nrm[q] += W[i * ka + q] * BW[i * ka + q];
            for (int q = 0; q < ka; ++q) nrm[q] = nrm[q] > 0 ? 1.0 / std::sqrt(nrm[q]) : 0.0;
            for (int64_t i = 0; i < m; ++i)
                for (int q = 0; q < ka; ++q) {
                    W[i * ka + q] *= nrm[q];
                    BW[i * ka + q] *= nrm[q];
                }
        }
        arrow_apply(A, ka, W.data(), AW.data());
        // basis S = [X, W, P]
        const int ns = k + ka + np;
        std::vector<double> S((size_t)m * ns), AS((size_t)m * ns), BS((size_t)m * ns);
        for (int64_t i = 0; i < m; ++i) {
            for (int j = 0; j < k; ++j) {
                S[i * ns + j] = X[i * k + j];
                AS[i * ns + j] = AX[i * k + j];
                BS[i * ns + j] = BX[i * k + j];
            }
            for (int q = 0; q < ka; ++q) {
                S[i * ns + k + q] = W[i * ka + q];
                AS[i * ns + k + q] = AW[i * ka + q];
                BS[i * ns + k + q] = BW[i * ka + q];
            }
            for (int q = 0; q < np; ++q) {
                S[i * ns + k + ka + q] = P[i * np + q];
                AS[i * ns + k + ka + q] = AP[i * np + q];
                BS[i * ns + k + ka + q] = BP[i * np + q];
            }
        }
        if (rayleigh_ritz(m, ns, S.data(), AS.data(), BS.data(), k, Y, theta) != 0) {
            if (np == 0) return -1;
            np = 0;  // restart without P
            continue;
        }
        // new X = S Y (products recomputed exactly); new P = (W, P) part of S Y, active columns
        mult(m, ns, S.data(), k, Y.data(), X.data());
        refresh();
        std::vector<double> Yp((size_t)ns * ka, 0.0);
        for (int a = k; a < ns; ++a)
            for (int q = 0; q < ka; ++q) Yp[a * ka + q] = Y[a * k + act[q]];
        P.assign((size_t)m * ka, 0.0);
        AP.assign((size_t)m * ka, 0.0);
        BP.assign((size_t)m * ka, 0.0);
        mult(m, ns, S.data(), ka, Yp.data(), P.data());
        np = ka;
        // exact images of P (implicitly updated images drift and break the Rayleigh-Ritz)
        arrow_apply(A, np, P.data(), AP.data());
        arrow_apply(B, np, P.data(), BP.data());
        {
            std::vector<double> nrm(np, 0.0);
            for (int64_t i = 0; i < m; ++i)
                for (int q = 0; q < np; ++q) nrm[q] += P[i * np + q] * BP[i * np + q];
            for (int q = 0; q < np; ++q) nrm[q] = nrm[q] > 0 ? 1.0 / std::sqrt(nrm[q]) : 0.0;
            for (int64_t i = 0; i < m; ++i)
                for (int q = 0; q < np; ++q) {
                    P[i * np + q] *= nrm[q];
                    AP[i * np + q] *= nrm[q];
                    BP[i * np + q] *= nrm[q];
                }
        }
    }
    if (it >= maxit) return -1;
    // final Rayleigh-Ritz within span X for B-orthonormal output
    if (rayleigh_ritz(m, k, X.data(), AX.data(), BX.data(), k, Y, theta) != 0) return -1;
    std::vector<double> Xf((size_t)m * k);
    mult(m, k, X.data(), k, Y.data(), Xf.data());
    for (int j = 0; j < nev; ++j) lam[j] = theta[j];
    for (int64_t i = 0; i < m; ++i)
        for (int j = 0; j < nev; ++j) U[i * nev + j] = Xf[i * k + j];
    return it;
}

}  // namespace nas
