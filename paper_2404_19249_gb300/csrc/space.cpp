// Host topology of P1/P2 spaces (see space.h).
#include "space.h"

#include <algorithm>
#include <string>

#include "common.h"

namespace nas {

static const int kEdges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

void build_space(HostSpace& S, int order, int64_t nv, const double* xyz, int64_t ne,
                 const int32_t* tet, bool with_patterns) {
    if (order != 1 && order != 2) fail(NAS_E_INVALID_ARG, "order must be 1 or 2");
    if (nv < 4 || ne < 1 || !xyz || !tet) fail(NAS_E_INVALID_ARG, "empty mesh");
    if (ne * 100 >= (int64_t)2147483647) fail(NAS_E_INVALID_ARG, "mesh too large for int32 slot lists");
    S = HostSpace();
    S.order = order;
    S.nloc = order == 1 ? 4 : 10;
    S.nv = nv;
    S.ne = ne;
    S.vxyz.assign(xyz, xyz + 3 * nv);
    for (int64_t i = 0; i < 4 * ne; ++i)
        if (tet[i] < 0 || tet[i] >= nv) fail(NAS_E_MESH, "tetrahedron vertex id out of range");
    for (int d = 0; d < 3; ++d) {
        S.lo[d] = S.hi[d] = xyz[d];
    }
    for (int64_t v = 0; v < nv; ++v)
        for (int d = 0; d < 3; ++d) {
            S.lo[d] = std::min(S.lo[d], xyz[3 * v + d]);
            S.hi[d] = std::max(S.hi[d], xyz[3 * v + d]);
        }

    const int nloc = S.nloc;
    S.elem.resize(ne * nloc);
    if (order == 1) {
        std::copy(tet, tet + 4 * ne, S.elem.begin());
        S.nnode = nv;
        S.node_xyz = S.vxyz;
    } else {
        // edges ordered by (smaller, larger) vertex id
        std::vector<int64_t> keys(ne * 6);
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < ne; ++e)
            for (int k = 0; k < 6; ++k) {
                int64_t a = tet[4 * e + kEdges[k][0]], b = tet[4 * e + kEdges[k][1]];
                if (a > b) std::swap(a, b);
                keys[e * 6 + k] = a * nv + b;
            }
        std::vector<int64_t> ukeys(keys);
        std::sort(ukeys.begin(), ukeys.end());
        ukeys.erase(std::unique(ukeys.begin(), ukeys.end()), ukeys.end());
        const int64_t nedge = (int64_t)ukeys.size();
        S.nnode = nv + nedge;
        if (S.nnode >= (int64_t)2147483647) fail(NAS_E_INVALID_ARG, "too many nodes");
        S.node_xyz.resize(3 * S.nnode);
        std::copy(xyz, xyz + 3 * nv, S.node_xyz.begin());
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nedge; ++k) {
            int64_t a = ukeys[k] / nv, b = ukeys[k] % nv;
            for (int d = 0; d < 3; ++d)
                S.node_xyz[3 * (nv + k) + d] = 0.5 * (xyz[3 * a + d] + xyz[3 * b + d]);
        }
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < ne; ++e) {
            for (int k = 0; k < 4; ++k) S.elem[e * 10 + k] = tet[4 * e + k];
            for (int k = 0; k < 6; ++k) {
                int64_t id = std::lower_bound(ukeys.begin(), ukeys.end(), keys[e * 6 + k]) - ukeys.begin();
                S.elem[e * 10 + 4 + k] = (int32_t)(nv + id);
            }
        }
    }

    // boundary = on a face of the vertices' bounding box (exact comparison)
    S.dof_of_node.assign(S.nnode, -1);
    S.bidx_of_node.assign(S.nnode, -1);
    for (int64_t u = 0; u < S.nnode; ++u) {
        bool b = false;
        for (int d = 0; d < 3; ++d) {
            double x = S.node_xyz[3 * u + d];
            if (x == S.lo[d] || x == S.hi[d]) b = true;
        }
        if (b) {
            S.bidx_of_node[u] = (int32_t)S.nb++;
            S.bnd_node.push_back((int32_t)u);
        } else {
            S.dof_of_node[u] = (int32_t)S.n++;
            S.dof_node.push_back((int32_t)u);
        }
    }
    if (S.n == 0) fail(NAS_E_MESH, "mesh has no interior nodes");
    if (!with_patterns) return;

    // node -> (element, local index) occurrences, ordered by element id
    std::vector<int64_t> aptr(S.nnode + 1, 0);
    for (int64_t i = 0; i < ne * nloc; ++i) aptr[S.elem[i] + 1]++;
    for (int64_t u = 0; u < S.nnode; ++u) aptr[u + 1] += aptr[u];
    std::vector<int32_t> adj(ne * nloc);
    {
        std::vector<int64_t> fill(aptr.begin(), aptr.end() - 1);
        for (int64_t i = 0; i < ne * nloc; ++i) adj[fill[S.elem[i]]++] = (int32_t)i;  // i = e*nloc + a
    }

    // load-vector lists of the interior dofs
    S.lptr.assign(S.n + 1, 0);
    for (int64_t d = 0; d < S.n; ++d) {
        int u = S.dof_node[d];
        S.lptr[d + 1] = S.lptr[d] + (aptr[u + 1] - aptr[u]);
    }
    S.lcontrib.resize(S.lptr[S.n]);
#pragma omp parallel for schedule(static)
    for (int64_t d = 0; d < S.n; ++d) {
        int u = S.dof_node[d];
        std::copy(adj.begin() + aptr[u], adj.begin() + aptr[u + 1], S.lcontrib.begin() + S.lptr[d]);
    }

    // CSR patterns with contribution lists, two passes (count, fill)
    const int64_t n = S.n;
    std::vector<int32_t> rnnz(n), rnnzb(n);
    std::vector<int64_t> rcon(n), rconb(n);
    auto row_pairs = [&](int64_t d, std::vector<std::pair<int32_t, int32_t>>& in,
                         std::vector<std::pair<int32_t, int32_t>>& bd) {
        in.clear();
        bd.clear();
        int u = S.dof_node[d];
        for (int64_t k = aptr[u]; k < aptr[u + 1]; ++k) {
            int64_t ea = adj[k];
            int64_t e = ea / nloc;
            for (int b = 0; b < nloc; ++b) {
                int v = S.elem[e * nloc + b];
                int32_t flat = (int32_t)(ea * nloc + b);
                if (S.dof_of_node[v] >= 0)
                    in.emplace_back(S.dof_of_node[v], flat);
                else
                    bd.emplace_back(S.bidx_of_node[v], flat);
            }
        }
        std::sort(in.begin(), in.end());
        std::sort(bd.begin(), bd.end());
    };
    auto count_unique = [](const std::vector<std::pair<int32_t, int32_t>>& v) {
        int32_t c = 0;
        for (size_t i = 0; i < v.size(); ++i)
            if (i == 0 || v[i].first != v[i - 1].first) ++c;
        return c;
    };
#pragma omp parallel
    {
        std::vector<std::pair<int32_t, int32_t>> in, bd;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t d = 0; d < n; ++d) {
            row_pairs(d, in, bd);
            rnnz[d] = count_unique(in);
            rnnzb[d] = count_unique(bd);
            rcon[d] = (int64_t)in.size();
            rconb[d] = (int64_t)bd.size();
        }
    }
    S.rowptr.assign(n + 1, 0);
    S.browptr.assign(n + 1, 0);
    std::vector<int64_t> cstart(n + 1, 0), bcstart(n + 1, 0);
    for (int64_t d = 0; d < n; ++d) {
        int64_t r = (int64_t)S.rowptr[d] + rnnz[d];
        if (r >= (int64_t)2147483647) fail(NAS_E_INVALID_ARG, "nnz exceeds int32");
        S.rowptr[d + 1] = (int32_t)r;
        S.browptr[d + 1] = S.browptr[d] + rnnzb[d];
        cstart[d + 1] = cstart[d] + rcon[d];
        bcstart[d + 1] = bcstart[d] + rconb[d];
    }
    S.col.resize(S.rowptr[n]);
    S.cptr.resize(S.rowptr[n] + 1);
    S.contrib.resize(cstart[n]);
    S.bcol.resize(S.browptr[n]);
    S.bcptr.resize(S.browptr[n] + 1);
    S.bcontrib.resize(bcstart[n]);
#pragma omp parallel
    {
        std::vector<std::pair<int32_t, int32_t>> in, bd;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t d = 0; d < n; ++d) {
            row_pairs(d, in, bd);
            int64_t s = S.rowptr[d] - 1, c = cstart[d];
            for (size_t i = 0; i < in.size(); ++i) {
                if (i == 0 || in[i].first != in[i - 1].first) {
                    ++s;
                    S.col[s] = in[i].first;
                    S.cptr[s] = c;
                }
                S.contrib[c++] = in[i].second;
            }
            s = S.browptr[d] - 1;
            c = bcstart[d];
            for (size_t i = 0; i < bd.size(); ++i) {
                if (i == 0 || bd[i].first != bd[i - 1].first) {
                    ++s;
                    S.bcol[s] = bd[i].first;
                    S.bcptr[s] = c;
                }
                S.bcontrib[c++] = bd[i].second;
            }
        }
    }
    S.cptr[S.rowptr[n]] = cstart[n];
    S.bcptr[S.browptr[n]] = bcstart[n];
}

}  // namespace nas
