// Point location of fine nodes in the nonnested coarse mesh, giving the
// transfer matrix I_H^h of Sec. 3.2 / Algorithm 1, as used in A_H = I^T A_h I of Sec. 3.3.
//
// GPU design: instead of Algorithm 1's octree + walk (a serial, branchy
// search), every fine node is one thread that reads the candidate coarse
// tetrahedra of its cell in a uniform bucket grid (each coarse tetrahedron is
// registered in every bucket its bounding box meets) and keeps the smallest
// element id whose CLOSED tetrahedron contains the node.  Containment is
// decided exactly: a floating-point orientation determinant with a forward
// error bound, and, when the bound cannot decide, an exact evaluation with
// floating-point expansions (error-free transformations: two-sum and the
// FMA-based two-product; expansions stay non-overlapping, so the sign is the
// sign of the last non-zero component).  Weights are D_k / D in floating
// point, D_k the orientation determinant with vertex k replaced by the node,
// set to exactly 0 where the exact sign is 0.
#include "kernels.h"

namespace nas {

// ---------------------------------------------------------------- error-free transforms
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    double aa = __dsub_rn(s, bb);
    e = __dadd_rn(__dsub_rn(a, aa), __dsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
    p = __dmul_rn(a, b);
    e = __fma_rn(a, b, -p);
}

// Grow-Expansion with zero elimination: e (length m, non-overlapping,
// increasing magnitude) += b.  Returns the new length.
__device__ int grow(double* e, int m, double b) {
    double q = b;
    int k = 0;
    for (int i = 0; i < m; ++i) {
        double s, h;
        two_sum(q, e[i], s, h);
        q = s;
        if (h != 0.0) e[k++] = h;
    }
    if (q != 0.0) e[k++] = q;
    return k;
}

// e += sign * a * b * c (exactly), a product of three doubles is 4 terms
__device__ int add_triple(double* e, int m, double a, double b, double c, double sign) {
    double p, pe;
    two_prod(b, c, p, pe);
    double t0, t0e, t1, t1e;
    two_prod(a, p, t0, t0e);
    two_prod(a, pe, t1, t1e);
    m = grow(e, m, sign * t1e);
    m = grow(e, m, sign * t1);
    m = grow(e, m, sign * t0e);
    m = grow(e, m, sign * t0);
    return m;
}

// e += sign * det3(p, q, r) with rows p, q, r (raw coordinates)
__device__ int add_det3(double* e, int m, const double* p, const double* q, const double* r, double sign) {
    m = add_triple(e, m, p[0], q[1], r[2], sign);
    m = add_triple(e, m, p[0], q[2], r[1], -sign);
    m = add_triple(e, m, p[1], q[2], r[0], sign);
    m = add_triple(e, m, p[1], q[0], r[2], -sign);
    m = add_triple(e, m, p[2], q[0], r[1], sign);
    m = add_triple(e, m, p[2], q[1], r[0], -sign);
    return m;
}

// Exact sign of det[b-a, c-a, d-a] = det3(b,c,d) - det3(a,c,d) + det3(a,b,d) - det3(a,b,c)
__device__ int orient_exact(const double* a, const double* b, const double* c, const double* d) {
    double e[112];
    int m = 0;
    m = add_det3(e, m, b, c, d, 1.0);
    m = add_det3(e, m, a, c, d, -1.0);
    m = add_det3(e, m, a, b, d, 1.0);
    m = add_det3(e, m, a, b, c, -1.0);
    if (m == 0) return 0;
    return e[m - 1] > 0.0 ? 1 : -1;
}

// Floating-point det[b-a, c-a, d-a] and a bound on its rounding error, with
// every operation rounded separately (no contraction) so the bound holds.
__device__ __forceinline__ double orient_float(const double* a, const double* b, const double* c,
                                               const double* d, double& err) {
    double bx = __dsub_rn(b[0], a[0]), by = __dsub_rn(b[1], a[1]), bz = __dsub_rn(b[2], a[2]);
    double cx = __dsub_rn(c[0], a[0]), cy = __dsub_rn(c[1], a[1]), cz = __dsub_rn(c[2], a[2]);
    double dx = __dsub_rn(d[0], a[0]), dy = __dsub_rn(d[1], a[1]), dz = __dsub_rn(d[2], a[2]);
    double m1 = __dsub_rn(__dmul_rn(cy, dz), __dmul_rn(cz, dy));
    double m2 = __dsub_rn(__dmul_rn(cx, dz), __dmul_rn(cz, dx));
    double m3 = __dsub_rn(__dmul_rn(cx, dy), __dmul_rn(cy, dx));
    double det = __dadd_rn(__dsub_rn(__dmul_rn(bx, m1), __dmul_rn(by, m2)), __dmul_rn(bz, m3));
    double p1 = __dadd_rn(__dmul_rn(fabs(cy), fabs(dz)), __dmul_rn(fabs(cz), fabs(dy)));
    double p2 = __dadd_rn(__dmul_rn(fabs(cx), fabs(dz)), __dmul_rn(fabs(cz), fabs(dx)));
    double p3 = __dadd_rn(__dmul_rn(fabs(cx), fabs(dy)), __dmul_rn(fabs(cy), fabs(dx)));
    double perm = __dadd_rn(__dadd_rn(__dmul_rn(fabs(bx), p1), __dmul_rn(fabs(by), p2)),
                            __dmul_rn(fabs(bz), p3));
    err = __dmul_rn(16.0 * 1.1102230246251565e-16, perm);
    return det;
}

__device__ __forceinline__ int orient_sign(const double* a, const double* b, const double* c,
                                           const double* d, double& det) {
    double err;
    det = orient_float(a, b, c, d, err);
    if (det > err) return 1;
    if (det < -err) return -1;
    return orient_exact(a, b, c, d);
}

// D_k signs of point p in tetrahedron V; returns true if all >= 0.
__device__ bool closed_contains(const double* p, const double V[4][3], int s[4], double dk[4]) {
    const double* W[4];
    for (int k = 0; k < 4; ++k) {
        for (int j = 0; j < 4; ++j) W[j] = (j == k) ? p : V[j];
        s[k] = orient_sign(W[0], W[1], W[2], W[3], dk[k]);
        if (s[k] < 0) return false;
    }
    return true;
}

// Bucket index of coordinate x: floor((x - org) * inv_h) clamped to [0, nb-1].
// The host registers tetrahedra with the same expression, rounded the same way.
__device__ __forceinline__ int bucket_of(double x, double org, double inv_h, int nb) {
    double t = __dmul_rn(__dsub_rn(x, org), inv_h);
    int b = (int)floor(t);
    return b < 0 ? 0 : (b >= nb ? nb - 1 : b);
}

__global__ void k_locate(LocateArgs a) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_points) return;
    const int node = a.point_node[i];
    double p[3] = {a.point_xyz[3 * node], a.point_xyz[3 * node + 1], a.point_xyz[3 * node + 2]};
    int bx = bucket_of(p[0], a.org[0], a.inv_h[0], a.nb[0]);
    int by = bucket_of(p[1], a.org[1], a.inv_h[1], a.nb[1]);
    int bz = bucket_of(p[2], a.org[2], a.inv_h[2], a.nb[2]);
    int64_t bucket = bx + (int64_t)a.nb[0] * (by + (int64_t)a.nb[1] * bz);
    int found = -1;
    int s[4];
    double dk[4];
    double V[4][3];
    for (int64_t k = a.bptr[bucket]; k < a.bptr[bucket + 1]; ++k) {
        int t = a.btet[k];  // ascending within the bucket: the first hit is the smallest id
        for (int j = 0; j < 4; ++j) {
            int v = a.ctet[4 * t + j];
            V[j][0] = a.cxyz[3 * v];
            V[j][1] = a.cxyz[3 * v + 1];
            V[j][2] = a.cxyz[3 * v + 2];
        }
        if (closed_contains(p, V, s, dk)) {
            found = t;
            break;
        }
    }
    a.elem[i] = found;
    if (found < 0) {
        atomicExch(a.error_flag, 1);
        for (int j = 0; j < 4; ++j) {
            a.icol[4 * i + j] = -1;
            a.ival[4 * i + j] = 0.0;
        }
        return;
    }
    double err;
    double D = orient_float(V[0], V[1], V[2], V[3], err);
    for (int j = 0; j < 4; ++j) {
        int v = a.ctet[4 * found + j];
        a.icol[4 * i + j] = a.coarse_dof_of_node[v];
        a.ival[4 * i + j] = (s[j] == 0) ? 0.0 : dk[j] / D;
    }
}

void launch_locate(const LocateArgs& a, cudaStream_t s) {
    if (a.n_points == 0) return;
    k_locate<<<grid_for(a.n_points, 128), 128, 0, s>>>(a);
    NAS_CHECK_LAUNCH();
}

}  // namespace nas
