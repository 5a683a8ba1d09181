// Host-side topology of a Lagrange P1/P2 space on a tetrahedral mesh:
// node numbering, boundary/interior split, CSR patterns and the gather lists
// that let the GPU assemble matrices deterministically (each CSR value is the
// sum, in a fixed order, of entries of element matrices).
#pragma once

#include <cstdint>
#include <vector>

namespace nas {

struct HostSpace {
    int order = 1;
    int nloc = 4;             // local nodes per element (4 or 10)
    int64_t nv = 0, ne = 0;   // vertices, elements
    int64_t nnode = 0;        // Lagrange nodes (vertices + edges for P2)
    int64_t n = 0;            // interior nodes = degrees of freedom
    int64_t nb = 0;           // boundary nodes
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // bounding box of the vertices

    std::vector<double> vxyz;          // [nv][3]
    std::vector<int32_t> elem;         // [ne][nloc] node ids
    std::vector<double> node_xyz;      // [nnode][3]
    std::vector<int32_t> dof_of_node;  // [nnode] dof or -1
    std::vector<int32_t> bidx_of_node; // [nnode] boundary index or -1
    std::vector<int32_t> dof_node;     // [n]  node of each dof
    std::vector<int32_t> bnd_node;     // [nb] node of each boundary index

    // interior x interior CSR pattern; value of slot s =
    //   sum_{k in [cptr[s], cptr[s+1])} Lbuf[contrib[k]]
    // with Lbuf the element matrices [ne][nloc][nloc] (flat index e*nloc^2+a*nloc+b)
    std::vector<int32_t> rowptr, col;
    std::vector<int64_t> cptr;
    std::vector<int32_t> contrib;
    // interior rows x boundary columns (Dirichlet lift), same scheme
    std::vector<int32_t> browptr, bcol;
    std::vector<int64_t> bcptr;
    std::vector<int32_t> bcontrib;
    // load vectors: b[dof] = sum_{k in [lptr[dof], lptr[dof+1])} Lvec[lcontrib[k]]
    // with Lvec the element vectors [ne][nloc] (flat index e*nloc+a)
    std::vector<int64_t> lptr;
    std::vector<int32_t> lcontrib;

    int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
    int64_t nnzb() const { return browptr.empty() ? 0 : browptr.back(); }
};

// Build the topology; throws nas::Error(NAS_E_MESH) on bad input.
// with_patterns = false skips the CSR patterns (coarse meshes only need the
// node numbering).
void build_space(HostSpace& S, int order, int64_t nv, const double* xyz, int64_t ne,
                 const int32_t* tet, bool with_patterns);

}  // namespace nas
