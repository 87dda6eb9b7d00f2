// Build-phase device routines (mesh, assembly, load vector, trees, A_H fill).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace hlu {

// A tetrahedral mesh on the device: the Kuhn cube (n > 0, vertices and
// tetrahedra implied by the lattice) or a general mesh (n == 0, vertex
// coordinates and tetrahedra stored).
struct DevMesh {
  int n = 0;
  int64_t N = 0;
  int32_t* dofmap = nullptr;  // lattice: (n+1)^3 x 7: DOF of edge (v, v + dir) or -1
  int32_t* edges = nullptr;   // N x 2 (lo, hi)
  int32_t* pts = nullptr;     // N x 3 tree points (lattice: doubled midpoints;
                              // general: quantized midpoints)
  int64_t nt = 0;             // tetrahedra
  int32_t nv = 0;             // vertices
  double* xyz = nullptr;      // general: nv x 3 coordinates
  int32_t* tets = nullptr;    // general: nt x 4 vertex ids
  int64_t* ekeys = nullptr;   // general: N interior-edge keys lo * nv + hi, ascending (DOF order)
  double* beta = nullptr;     // material coefficient per tetrahedron (null: 1)
};
struct DevCSR {
  int64_t N = 0, nnz = 0;
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};
struct HostTrees {
  int32_t nc = 0, nb = 0;
  std::vector<int32_t> clusters;  // nc x 12 export layout
  std::vector<int32_t> blocks;    // nb x 8 export layout
  std::vector<int32_t> perm;      // N
};
// A_H fill descriptor of one leaf block.
struct FillDesc {
  int64_t off;         // dense storage or X storage (elements)
  int64_t off2;        // Y storage (admissible)
  int64_t row_prefix;  // dense: rows of all earlier dense descriptors
  int32_t roff, m, coff, n;
  int32_t slot, cap;
};

cudaError_t build_mesh_dofs(int n, cudaStream_t s, DevMesh& m);
// General mesh: xyz (nv x 3) and tets (nt x 4, ids in [0, nv)) on the host.
// Interior edges (edges on no boundary face; a boundary face belongs to one
// tetrahedron) numbered in (lo, hi) order; tree points p = rint((x_lo + x_hi
// - 2 lo_box) s) with s the largest power of two keeping them <= 2^21.
cudaError_t build_mesh_general(int32_t nv, int64_t nt, const double* xyz, const int32_t* tets, cudaStream_t s,
                               DevMesh& m);
cudaError_t assemble_csr(const DevMesh& m, double kappa, cudaStream_t s, DevCSR& A);
cudaError_t manufactured_rhs(const DevMesh& m, double kappa, double* b, cudaStream_t s);
// load vector of the constant current density J (exact integration)
cudaError_t constant_current_rhs(const DevMesh& m, const double J[3], double* b, cudaStream_t s);
// manufactured_rhs without allocations (fixed device scratch; see build.cu);
// cudaErrorInvalidValue when the mesh needs more than rhs_noalloc_max_entries()
// element contributions
cudaError_t manufactured_rhs_noalloc(const DevMesh& m, double kappa, double* b, cudaStream_t s);
int64_t rhs_noalloc_max_entries();
cudaError_t build_trees(const DevMesh& m, int32_t leaf, int64_t eta2, cudaStream_t s, HostTrees& out,
                        int32_t* d_perm_out);
cudaError_t invert_perm(int32_t N, const int32_t* perm, int32_t* iperm, cudaStream_t s);
template <class T>
cudaError_t fill_ah(const DevCSR& A, const int32_t* d_perm, const int32_t* d_iperm, const FillDesc* d_dense,
                    int32_t ndense, int64_t dense_rows, const FillDesc* d_lr, int32_t nlr, T* arena,
                    int64_t zero_elems, int64_t ident_off, int32_t ident_n, int32_t* ranks, int32_t* status,
                    cudaStream_t s);

}  // namespace hlu
