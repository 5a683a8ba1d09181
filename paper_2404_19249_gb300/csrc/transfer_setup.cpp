// Host-side transfer structures (see transfer_setup.h).
#include "transfer_setup.h"

#include <algorithm>
#include <cmath>

#include "common.h"

namespace nas {

static inline int bucket_of(double x, double org, double inv_h, int nb) {
    // Same expression and rounding as the device side: floor((x - org) * inv_h)
    volatile double d = x - org;
    volatile double t = d * inv_h;
    int b = (int)std::floor(t);
    return b < 0 ? 0 : (b >= nb ? nb - 1 : b);
}

void build_buckets(const HostSpace& C, BucketGrid& G) {
    const int64_t nt = C.ne;
    int per = (int)std::ceil(std::cbrt((double)nt / 2.0));
    per = std::max(1, std::min(per, 256));
    for (int d = 0; d < 3; ++d) {
        G.nb[d] = per;
        G.org[d] = C.lo[d];
        double w = C.hi[d] - C.lo[d];
        G.inv_h[d] = w > 0 ? per / w : 1.0;
    }
    const int64_t nbk = (int64_t)G.nb[0] * G.nb[1] * G.nb[2];
    std::vector<int32_t> lo(nt * 3), hi(nt * 3);
    for (int64_t t = 0; t < nt; ++t) {
        for (int d = 0; d < 3; ++d) {
            double mn = 1e300, mx = -1e300;
            for (int k = 0; k < 4; ++k) {
                double x = C.vxyz[3 * C.elem[4 * t + k] + d];
                mn = std::min(mn, x);
                mx = std::max(mx, x);
            }
            lo[3 * t + d] = bucket_of(mn, G.org[d], G.inv_h[d], G.nb[d]);
            hi[3 * t + d] = bucket_of(mx, G.org[d], G.inv_h[d], G.nb[d]);
        }
    }
    G.bptr.assign(nbk + 1, 0);
    for (int64_t t = 0; t < nt; ++t)
        for (int z = lo[3 * t + 2]; z <= hi[3 * t + 2]; ++z)
            for (int y = lo[3 * t + 1]; y <= hi[3 * t + 1]; ++y)
                for (int x = lo[3 * t]; x <= hi[3 * t]; ++x)
                    G.bptr[x + (int64_t)G.nb[0] * (y + (int64_t)G.nb[1] * z) + 1]++;
    for (int64_t b = 0; b < nbk; ++b) G.bptr[b + 1] += G.bptr[b];
    G.btet.resize(G.bptr[nbk]);
    std::vector<int64_t> fill(G.bptr.begin(), G.bptr.end() - 1);
    for (int64_t t = 0; t < nt; ++t)  // ascending t: lists come out sorted
        for (int z = lo[3 * t + 2]; z <= hi[3 * t + 2]; ++z)
            for (int y = lo[3 * t + 1]; y <= hi[3 * t + 1]; ++y)
                for (int x = lo[3 * t]; x <= hi[3 * t]; ++x)
                    G.btet[fill[x + (int64_t)G.nb[0] * (y + (int64_t)G.nb[1] * z)]++] = (int32_t)t;
}

void build_galerkin(const HostSpace& F, int64_t nH, const std::vector<int32_t>& icol,
                    const std::vector<double>& ival, GalerkinMaps& G) {
    const int64_t n = F.n;
    G = GalerkinMaps();
    G.nH = nH;
    // ---- I^T
    G.tptr.assign(nH + 1, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 4; ++k)
            if (icol[4 * i + k] >= 0) G.tptr[icol[4 * i + k] + 1]++;
    for (int64_t a = 0; a < nH; ++a) G.tptr[a + 1] += G.tptr[a];
    G.trow.resize(G.tptr[nH]);
    G.tval.resize(G.tptr[nH]);
    {
        std::vector<int64_t> fill(G.tptr.begin(), G.tptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 4; ++k) {
                int a = icol[4 * i + k];
                if (a < 0) continue;
                G.trow[fill[a]] = (int32_t)i;
                G.tval[fill[a]++] = ival[4 * i + k];
            }
    }
    // ---- W = A I pattern and stage-1 lists (two passes over the fine rows)
    std::vector<int32_t> wn(n);
    std::vector<int64_t> wc(n);
    auto wpairs = [&](int64_t i, std::vector<std::pair<int32_t, int32_t>>& v) {
        v.clear();
        for (int p = F.rowptr[i]; p < F.rowptr[i + 1]; ++p) {
            int j = F.col[p];
            for (int l = 0; l < 4; ++l) {
                int b = icol[4 * (int64_t)j + l];
                if (b >= 0) v.emplace_back(b, (int32_t)(4 * (int64_t)p + l));
            }
        }
        std::sort(v.begin(), v.end());
    };
#pragma omp parallel
    {
        std::vector<std::pair<int32_t, int32_t>> v;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) {
            wpairs(i, v);
            int32_t u = 0;
            for (size_t k = 0; k < v.size(); ++k)
                if (k == 0 || v[k].first != v[k - 1].first) ++u;
            wn[i] = u;
            wc[i] = (int64_t)v.size();
        }
    }
    G.wptr.assign(n + 1, 0);
    std::vector<int64_t> cst(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = (int64_t)G.wptr[i] + wn[i];
        if (r >= (int64_t)2147483647 / 4) fail(NAS_E_INVALID_ARG, "transfer product too large for int32 lists");
        G.wptr[i + 1] = (int32_t)r;
        cst[i + 1] = cst[i] + wc[i];
    }
    const int64_t wnnz = G.wptr[n];
    G.wcol.resize(wnnz);
    G.wrow.resize(wnnz);
    G.w1ptr.resize(wnnz + 1);
    G.w1con.resize(cst[n]);
#pragma omp parallel
    {
        std::vector<std::pair<int32_t, int32_t>> v;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) {
            wpairs(i, v);
            int64_t s = G.wptr[i] - 1, c = cst[i];
            for (size_t k = 0; k < v.size(); ++k) {
                if (k == 0 || v[k].first != v[k - 1].first) {
                    ++s;
                    G.wcol[s] = v[k].first;
                    G.wrow[s] = (int32_t)i;
                    G.w1ptr[s] = c;
                }
                G.w1con[c++] = v[k].second;
            }
        }
    }
    G.w1ptr[wnnz] = cst[n];
    // ---- A_H pattern and stage-2 lists: coarse row a gathers over fine rows i
    // with I_ia != 0 (k = position of a in row i) and their W slots s
    std::vector<int32_t> hn(nH);
    std::vector<int64_t> hc(nH);
    auto hpairs = [&](int64_t a, std::vector<std::pair<int32_t, int32_t>>& v) {
        v.clear();
        for (int p = G.tptr[a]; p < G.tptr[a + 1]; ++p) {
            int64_t i = G.trow[p];
            int k = 0;
            while (k < 4 && icol[4 * i + k] != (int32_t)a) ++k;
            for (int s = G.wptr[i]; s < G.wptr[i + 1]; ++s)
                v.emplace_back(G.wcol[s], (int32_t)(4 * (int64_t)s + k));
        }
        std::sort(v.begin(), v.end());
    };
#pragma omp parallel
    {
        std::vector<std::pair<int32_t, int32_t>> v;
#pragma omp for schedule(dynamic, 1)
        for (int64_t a = 0; a < nH; ++a) {
            hpairs(a, v);
            int32_t u = 0;
            for (size_t k = 0; k < v.size(); ++k)
                if (k == 0 || v[k].first != v[k - 1].first) ++u;
            hn[a] = u;
            hc[a] = (int64_t)v.size();
        }
    }
    G.hptr.assign(nH + 1, 0);
    std::vector<int64_t> hst(nH + 1, 0);
    for (int64_t a = 0; a < nH; ++a) {
        G.hptr[a + 1] = G.hptr[a] + hn[a];
        hst[a + 1] = hst[a] + hc[a];
    }
    const int64_t hnnz = G.hptr[nH];
    G.hcol.resize(hnnz);
    G.h2ptr.resize(hnnz + 1);
    G.h2con.resize(hst[nH]);
#pragma omp parallel
    {
        std::vector<std::pair<int32_t, int32_t>> v;
#pragma omp for schedule(dynamic, 1)
        for (int64_t a = 0; a < nH; ++a) {
            hpairs(a, v);
            int64_t s = G.hptr[a] - 1, c = hst[a];
            for (size_t k = 0; k < v.size(); ++k) {
                if (k == 0 || v[k].first != v[k - 1].first) {
                    ++s;
                    G.hcol[s] = v[k].first;
                    G.h2ptr[s] = c;
                }
                G.h2con[c++] = v[k].second;
            }
        }
    }
    G.h2ptr[hnnz] = hst[nH];
    make_pieces(G.tptr, 128, G.tpieces);
    make_pieces(G.h2ptr, 256, G.h2pieces);
}

template <typename P>
void make_pieces(const std::vector<P>& ptr, int64_t len, PieceMap& pm) {
    const int64_t nseg = (int64_t)ptr.size() - 1;
    pm.seg_piece.assign(std::max<int64_t>(nseg, 0) + 1, 0);
    pm.piece_start.clear();
    for (int64_t a = 0; a < nseg; ++a) {
        const int64_t b = ptr[a], e = ptr[a + 1];
        const int64_t np = (e - b + len - 1) / len;
        if ((int64_t)pm.seg_piece[a] + np > 2147483647) fail(NAS_E_INVALID_ARG, "too many list pieces");
        for (int64_t q = 0; q < np; ++q) pm.piece_start.push_back(b + q * len);
        pm.seg_piece[a + 1] = pm.seg_piece[a] + (int32_t)np;
    }
    pm.piece_start.push_back(nseg > 0 ? (int64_t)ptr[nseg] : 0);
}
template void make_pieces<int32_t>(const std::vector<int32_t>&, int64_t, PieceMap&);
template void make_pieces<int64_t>(const std::vector<int64_t>&, int64_t, PieceMap&);

}  // namespace nas
