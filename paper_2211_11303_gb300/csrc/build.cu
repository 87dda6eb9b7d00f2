// Build-phase kernels (Algorithm 1 step I and the structures it needs):
//   * Kuhn-cube mesh and interior-edge DOF numbering (Sec. 2.1: one DOF per
//     interior edge, sigma(Phi_i, e_j) = delta_ij, boundary edges carry E x n = 0);
//   * FP64 assembly of A = K - kappa^2 M (Sec. 2.1 weak form and
//     stiffness-matrix equation) into CSR;
//   * load vector b_j = <J, Phi_j> of the manufactured field;
//   * geometric cluster tree (Sec. 4, geometrically balanced bisection) and the
//     eta-admissible block tree (Sec. 3-4), integer-exact, level by level;
//   * A_H: dense leaves and exact low-rank admissible blocks from the CSR matrix.
//
// Mesh readings: vertex (i,j,k) has id (i(n+1)+j)(n+1)+k; every Kuhn edge goes
// from a vertex v to v + d, d one of the 7 nonzero 0/1 vectors, so the edges
// sorted by (lo, hi) are enumerated vertex by vertex with d ordered by the id
// offset: 001, 010, 011, 100, 101, 110, 111.  An edge is a boundary edge iff
// some axis a has d_a = 0 and v_a in {0, n}.
#include <cuda_runtime.h>
#include <thrust/device_ptr.h>
#include <thrust/execution_policy.h>
#include <thrust/reduce.h>
#include <thrust/scan.h>
#include <thrust/sequence.h>
#include <thrust/fill.h>
#include <thrust/set_operations.h>
#include <thrust/sort.h>
#include <thrust/unique.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "launch_count.h"

#include "build.h"
#include "devmem.h"

namespace hlu {

__constant__ int c_dir[7][3] = {{0, 0, 1}, {0, 1, 0}, {0, 1, 1}, {1, 0, 0},
                                {1, 0, 1}, {1, 1, 0}, {1, 1, 1}};
// Kuhn tetrahedra: axis permutations in lexicographic order
__constant__ int c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
__constant__ int c_ledge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

__device__ __forceinline__ void vcoord(int64_t v, int n, int* p) {
  p[2] = (int)(v % (n + 1));
  v /= (n + 1);
  p[1] = (int)(v % (n + 1));
  p[0] = (int)(v / (n + 1));
}

// ---------------------------------------------------------------- DOFs
__global__ void k_count_edges(int n, int32_t* cnt) {
  int64_t nv = (int64_t)(n + 1) * (n + 1) * (n + 1);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    int p[3];
    vcoord(v, n, p);
    int c = 0;
    for (int d = 0; d < 7; ++d) {
      bool ok = true, bnd = false;
      for (int a = 0; a < 3; ++a) {
        if (p[a] + c_dir[d][a] > n) ok = false;
        if (c_dir[d][a] == 0 && (p[a] == 0 || p[a] == n)) bnd = true;
      }
      c += (ok && !bnd);
    }
    cnt[v] = c;
  }
}

__global__ void k_number_edges(int n, const int32_t* start, int32_t* dofmap, int32_t* edges, int32_t* pts) {
  int64_t nv = (int64_t)(n + 1) * (n + 1) * (n + 1);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    int p[3];
    vcoord(v, n, p);
    int32_t dof = start[v];
    for (int d = 0; d < 7; ++d) {
      bool ok = true, bnd = false;
      for (int a = 0; a < 3; ++a) {
        if (p[a] + c_dir[d][a] > n) ok = false;
        if (c_dir[d][a] == 0 && (p[a] == 0 || p[a] == n)) bnd = true;
      }
      if (ok && !bnd) {
        int64_t w = v + (int64_t)c_dir[d][0] * (n + 1) * (n + 1) + c_dir[d][1] * (n + 1) + c_dir[d][2];
        dofmap[v * 7 + d] = dof;
        edges[2 * (int64_t)dof] = (int32_t)v;
        edges[2 * (int64_t)dof + 1] = (int32_t)w;
        for (int a = 0; a < 3; ++a) pts[3 * (int64_t)dof + a] = 2 * p[a] + c_dir[d][a];
        ++dof;
      } else {
        dofmap[v * 7 + d] = -1;
      }
    }
  }
}

__device__ __forceinline__ int dir_index(int dx, int dy, int dz) {
  int code = dx * 4 + dy * 2 + dz;  // 1..7 -> index in c_dir order
  return code - 1;
}

struct TetGeo {
  int64_t v[4];
  double P[4][3];
  double G[4][3];
  double vol;
  int dof[6];
  int lo[6], hi[6];  // oriented local vertex pair of each local edge
};

__device__ void tet_geometry_lattice(int64_t t, int n, const int32_t* dofmap, TetGeo& g) {
  int64_t cube = t / 6;
  int pi = (int)(t % 6);
  int c[3];
  c[2] = (int)(cube % n);
  c[1] = (int)((cube / n) % n);
  c[0] = (int)(cube / ((int64_t)n * n));
  int p[3] = {c[0], c[1], c[2]};
  int L[4][3];
  for (int a = 0; a < 3; ++a) L[0][a] = p[a];
  for (int s = 0; s < 3; ++s) {
    for (int a = 0; a < 3; ++a) L[s + 1][a] = L[s][a];
    L[s + 1][c_perm[pi][s]] += 1;
  }
  for (int s = 0; s < 4; ++s) {
    g.v[s] = ((int64_t)L[s][0] * (n + 1) + L[s][1]) * (n + 1) + L[s][2];
    for (int a = 0; a < 3; ++a) g.P[s][a] = (double)L[s][a] / (double)n;
  }
  double J[3][3];
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 3; ++s) J[a][s] = g.P[s + 1][a] - g.P[0][a];  // columns p_s - p_0
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int a = 0; a < 3; ++a) {
    g.G[0][a] = 0;
    for (int s = 0; s < 3; ++s) {
      g.G[s + 1][a] = inv[s][a];  // rows of J^-1
      g.G[0][a] -= inv[s][a];
    }
  }
  g.vol = fabs(det) / 6.0;
  for (int e = 0; e < 6; ++e) {
    int a = c_ledge[e][0], b = c_ledge[e][1];
    if (g.v[a] > g.v[b]) {
      int tmp = a;
      a = b;
      b = tmp;
    }
    g.lo[e] = a;
    g.hi[e] = b;
    int d[3];
    for (int x = 0; x < 3; ++x) d[x] = L[b][x] - L[a][x];
    int di = dir_index(d[0], d[1], d[2]);
    g.dof[e] = (di >= 0 && di < 7) ? dofmap[g.v[a] * 7 + di] : -1;
  }
}

// What the element kernels read of a mesh (DevMesh without ownership).
struct MeshView {
  int n;            // lattice size, 0 for a general mesh
  int64_t nt;       // tetrahedra
  int32_t nv;
  const int32_t* dofmap;
  const double* xyz;
  const int32_t* tets;
  const int64_t* ekeys;
  int64_t N;
  const double* beta;  // material coefficient per tetrahedron (null: 1)
};
static MeshView view_of(const DevMesh& m) {
  return MeshView{m.n, m.n > 0 ? (int64_t)6 * m.n * m.n * m.n : m.nt, m.nv, m.dofmap, m.xyz, m.tets, m.ekeys, m.N,
                  m.beta};
}

// General tetrahedron t: coordinates from xyz, barycentric gradients as in
// the lattice case, local edge -> interior DOF by binary search of its key.
__device__ void tet_geometry_general(int64_t t, const MeshView& mv, TetGeo& g) {
  for (int s = 0; s < 4; ++s) {
    g.v[s] = mv.tets[4 * t + s];
    for (int a = 0; a < 3; ++a) g.P[s][a] = mv.xyz[3 * g.v[s] + a];
  }
  double J[3][3];
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 3; ++s) J[a][s] = g.P[s + 1][a] - g.P[0][a];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int a = 0; a < 3; ++a) {
    g.G[0][a] = 0;
    for (int s = 0; s < 3; ++s) {
      g.G[s + 1][a] = inv[s][a];
      g.G[0][a] -= inv[s][a];
    }
  }
  g.vol = fabs(det) / 6.0;
  for (int e = 0; e < 6; ++e) {
    int a = c_ledge[e][0], b = c_ledge[e][1];
    if (g.v[a] > g.v[b]) {
      int tmp = a;
      a = b;
      b = tmp;
    }
    g.lo[e] = a;
    g.hi[e] = b;
    const int64_t key = g.v[a] * (int64_t)mv.nv + g.v[b];
    int64_t lo = 0, hi = mv.N;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (mv.ekeys[mid] < key)
        lo = mid + 1;
      else
        hi = mid;
    }
    g.dof[e] = (lo < mv.N && mv.ekeys[lo] == key) ? (int)lo : -1;
  }
}

__device__ __forceinline__ void tet_geometry(int64_t t, const MeshView& mv, TetGeo& g) {
  if (mv.n > 0)
    tet_geometry_lattice(t, mv.n, mv.dofmap, g);
  else
    tet_geometry_general(t, mv, g);
}

__device__ __forceinline__ double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// one thread per tetrahedron: 36 (key, value) pairs, key = row * N + col or
// INT64_MAX for pairs that touch a boundary edge; the curl-curl part is
// divided by the element's material coefficient
__global__ void k_element_coo(MeshView mv, double kappa2, int64_t N, int64_t* keys, double* vals) {
  const int64_t nt = mv.nt;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    TetGeo g;
    tet_geometry(t, mv, g);
    const double ib = mv.beta ? 1.0 / mv.beta[t] : 1.0;
    for (int r = 0; r < 6; ++r) {
      int a = g.lo[r], b = g.hi[r];
      double ca[3];
      cross3(g.G[a], g.G[b], ca);
      for (int s = 0; s < 6; ++s) {
        int cc = g.lo[s], d = g.hi[s];
        double cb[3];
        cross3(g.G[cc], g.G[d], cb);
        double K = ib * (4.0 * g.vol * dot3(ca, cb));
        auto mom = [&](int i, int j) { return g.vol * (i == j ? 2.0 : 1.0) / 20.0; };
        double M = mom(a, cc) * dot3(g.G[b], g.G[d]) - mom(a, d) * dot3(g.G[b], g.G[cc]) -
                   mom(b, cc) * dot3(g.G[a], g.G[d]) + mom(b, d) * dot3(g.G[a], g.G[cc]);
        int64_t o = t * 36 + r * 6 + s;
        if (g.dof[r] >= 0 && g.dof[s] >= 0) {
          keys[o] = (int64_t)g.dof[r] * N + g.dof[s];
          vals[o] = K - kappa2 * M;
        } else {
          keys[o] = INT64_MAX;
          vals[o] = 0.0;
        }
      }
    }
  }
}

__global__ void k_csr_rows(int64_t nnz, int64_t N, const int64_t* ukeys, int32_t* col, int32_t* rowcnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = ukeys[e];
    col[e] = (int32_t)(k % N);
    atomicAdd(rowcnt + (k / N), 1);
  }
}

// load vector: one thread per tetrahedron, 6 (dof, value) pairs
__global__ void k_rhs_coo(MeshView mv, double kappa2, int32_t* keys, double* vals) {
  const int64_t nt = mv.nt;
  const double qa = (5.0 - sqrt(5.0)) / 20.0, qb = (5.0 + 3.0 * sqrt(5.0)) / 20.0;
  const double PI = 3.14159265358979323846;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    TetGeo g;
    tet_geometry(t, mv, g);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int q = 0; q < 4; ++q) {
      double lam[4] = {qa, qa, qa, qa};
      lam[q] = qb;
      double x[3] = {0, 0, 0};
      for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) x[a] += lam[s] * g.P[s][a];
      double sx = sin(PI * x[0]), sy = sin(PI * x[1]), sz = sin(PI * x[2]);
      double f = 2.0 * PI * PI - kappa2;
      double J[3] = {f * sy * sz, f * sz * sx, f * sx * sy};
      for (int e = 0; e < 6; ++e) {
        int a = g.lo[e], b = g.hi[e];
        double phi[3];
        for (int c = 0; c < 3; ++c) phi[c] = lam[a] * g.G[b][c] - lam[b] * g.G[a][c];
        acc[e] += dot3(J, phi);
      }
    }
    for (int e = 0; e < 6; ++e) {
      keys[t * 6 + e] = g.dof[e] >= 0 ? g.dof[e] : INT32_MAX;
      vals[t * 6 + e] = g.vol / 4.0 * acc[e];
    }
  }
}

// load vector of a constant current density J (Sec. 4, Example 1: J_S =
// [0, 0, 1]): Phi_ab = lam_a grad lam_b - lam_b grad lam_a is linear and the
// integral of a barycentric coordinate over T is |T| / 4, so
// b_e = |T| / 4 J . (grad lam_b - grad lam_a) exactly.  One thread per
// tetrahedron, 6 (dof, value) pairs.
__global__ void k_rhs_const_coo(MeshView mv, double J0, double J1, double J2, int32_t* keys, double* vals) {
  const int64_t nt = mv.nt;
  const double J[3] = {J0, J1, J2};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    TetGeo g;
    tet_geometry(t, mv, g);
    for (int e = 0; e < 6; ++e) {
      const int a = g.lo[e], b = g.hi[e];
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = g.G[b][c] - g.G[a][c];
      keys[t * 6 + e] = g.dof[e] >= 0 ? g.dof[e] : INT32_MAX;
      vals[t * 6 + e] = g.vol / 4.0 * dot3(J, d);
    }
  }
}

__global__ void k_scatter_rhs(int64_t m, const int32_t* ukeys, const double* sums, int64_t N, double* b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t k = ukeys[e];
    if (k >= 0 && k < N) b[k] = sums[e];
  }
}

// ---------------------------------------------------------------- cluster tree
// One CTA per cluster of the current level: tight bounding box of its points.
__global__ void k_cluster_bbox(int32_t nc, const int32_t* off, const int32_t* size, const int32_t* perm,
                               const int32_t* pts, int32_t* lo, int32_t* hi) {
  __shared__ int32_t s[6][32];
  for (int32_t c = blockIdx.x; c < nc; c += gridDim.x) {
    int32_t mn[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, mx[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int32_t i = threadIdx.x; i < size[c]; i += blockDim.x) {
      int32_t d = perm[off[c] + i];
      for (int a = 0; a < 3; ++a) {
        int32_t v = pts[3 * (int64_t)d + a];
        mn[a] = min(mn[a], v);
        mx[a] = max(mx[a], v);
      }
    }
    for (int a = 0; a < 3; ++a)
      for (int o = 16; o > 0; o >>= 1) {
        mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
        mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
      }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
      for (int a = 0; a < 3; ++a) {
        s[a][w] = mn[a];
        s[3 + a][w] = mx[a];
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int a = 0; a < 3; ++a) {
        int32_t m0 = INT32_MAX, m1 = INT32_MIN;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
          m0 = min(m0, s[a][k]);
          m1 = max(m1, s[3 + a][k]);
        }
        lo[3 * (int64_t)c + a] = size[c] ? m0 : 0;
        hi[3 * (int64_t)c + a] = size[c] ? m1 : 0;
      }
    }
    __syncthreads();
  }
}

// One CTA per cluster: stable partition by 2 p[ax] < lo[ax] + hi[ax] (leaves copy).
__global__ void k_cluster_split(int32_t nc, int32_t leaf, const int32_t* off, const int32_t* size, const int32_t* lo,
                                const int32_t* hi, const int32_t* perm_in, int32_t* perm_out, const int32_t* pts,
                                int32_t* nleft) {
  __shared__ int32_t s_scan[1024];
  __shared__ int32_t s_base[2];
  for (int32_t c = blockIdx.x; c < nc; c += gridDim.x) {
    const int32_t o = off[c], sz = size[c];
    if (sz <= leaf) {
      for (int32_t i = threadIdx.x; i < sz; i += blockDim.x) perm_out[o + i] = perm_in[o + i];
      if (threadIdx.x == 0) nleft[c] = -1;
      __syncthreads();
      continue;
    }
    int ax = 0;
    int32_t e0 = hi[3 * (int64_t)c] - lo[3 * (int64_t)c];
    for (int a = 1; a < 3; ++a) {
      int32_t e = hi[3 * (int64_t)c + a] - lo[3 * (int64_t)c + a];
      if (e > e0) {
        e0 = e;
        ax = a;
      }
    }
    const int32_t mid2 = lo[3 * (int64_t)c + ax] + hi[3 * (int64_t)c + ax];
    // count left points
    int32_t cntl = 0;
    for (int32_t i = threadIdx.x; i < sz; i += blockDim.x) cntl += (2 * pts[3 * (int64_t)perm_in[o + i] + ax] < mid2);
    s_scan[threadIdx.x] = cntl;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if ((int)threadIdx.x < st) s_scan[threadIdx.x] += s_scan[threadIdx.x + st];
      __syncthreads();
    }
    const int32_t total_left = s_scan[0];
    __syncthreads();
    if (threadIdx.x == 0) {
      s_base[0] = 0;
      s_base[1] = 0;
      nleft[c] = total_left;
    }
    __syncthreads();
    for (int32_t base = 0; base < sz; base += blockDim.x) {
      int32_t i = base + threadIdx.x;
      int32_t d = i < sz ? perm_in[o + i] : 0;
      int32_t f = (i < sz) && (2 * pts[3 * (int64_t)d + ax] < mid2);
      // inclusive scan of f over the block
      s_scan[threadIdx.x] = f;
      __syncthreads();
      for (int st = 1; st < (int)blockDim.x; st <<= 1) {
        int32_t v = (int)threadIdx.x >= st ? s_scan[threadIdx.x - st] : 0;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
      }
      int32_t incl = s_scan[threadIdx.x];
      int32_t chunk_left = s_scan[blockDim.x - 1];
      if (i < sz) {
        if (f)
          perm_out[o + s_base[0] + incl - 1] = d;
        else
          perm_out[o + total_left + s_base[1] + (threadIdx.x - incl)] = d;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int32_t nvalid = min((int32_t)blockDim.x, sz - base);
        s_base[0] += chunk_left;
        s_base[1] += nvalid - chunk_left;
      }
      __syncthreads();
    }
  }
}

// next level's clusters from the split results (single CTA, sequential scan)
__global__ void k_cluster_children(int32_t nc, int32_t first_id, const int32_t* off, const int32_t* size,
                                   const int32_t* nleft, int32_t* son, int32_t* noff, int32_t* nsize,
                                   int32_t* nparent, int32_t* count) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t k = 0;
  for (int32_t c = 0; c < nc; ++c) {
    if (nleft[c] <= 0 || nleft[c] >= size[c]) {  // leaf (or a degenerate box that cannot split)
      son[2 * c] = son[2 * c + 1] = -1;
      continue;
    }
    noff[k] = off[c];
    nsize[k] = nleft[c];
    nparent[k] = first_id + c;
    noff[k + 1] = off[c] + nleft[c];
    nsize[k + 1] = size[c] - nleft[c];
    nparent[k + 1] = first_id + c;
    son[2 * c] = k;
    son[2 * c + 1] = k + 1;
    k += 2;
  }
  *count = k;
}

// ---------------------------------------------------------------- block tree
__device__ __forceinline__ int64_t diam2(const int32_t* lo, const int32_t* hi, int32_t c) {
  int64_t s = 0;
  for (int a = 0; a < 3; ++a) {
    int64_t d = (int64_t)hi[3 * c + a] - lo[3 * c + a];
    s += d * d;
  }
  return s;
}
__device__ __forceinline__ int64_t dist2(const int32_t* lo, const int32_t* hi, int32_t t, int32_t s) {
  int64_t r = 0;
  for (int a = 0; a < 3; ++a) {
    int64_t g1 = (int64_t)lo[3 * s + a] - hi[3 * t + a];
    int64_t g2 = (int64_t)lo[3 * t + a] - hi[3 * s + a];
    int64_t g = g1 > g2 ? g1 : g2;
    if (g < 0) g = 0;
    r += g * g;
  }
  return r;
}

// classify the blocks of one level; sub-divided blocks count 4 children
__global__ void k_block_classify(int32_t nb, const int32_t* brow, const int32_t* bcol, const int32_t* clo,
                                 const int32_t* chi, const int32_t* cson, int64_t eta2, int32_t* kind,
                                 int32_t* nchild) {
  for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    int32_t t = brow[b], s = bcol[b];
    int64_t d2 = dist2(clo, chi, t, s);
    int64_t dm = min(diam2(clo, chi, t), diam2(clo, chi, s));
    int k;
    if (d2 > 0 && dm <= eta2 * d2)
      k = 0;
    else if (cson[2 * t] < 0 || cson[2 * s] < 0)
      k = 1;
    else
      k = 2;
    kind[b] = k;
    nchild[b] = k == 2 ? 4 : 0;
  }
}

__global__ void k_block_expand(int32_t nb, const int32_t* brow, const int32_t* bcol, const int32_t* kind,
                               const int32_t* cstart, const int32_t* cson, int32_t first_child_id,
                               int32_t first_id, int32_t* bson, int32_t* nrow, int32_t* ncol, int32_t* npar) {
  for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    if (kind[b] != 2) {
      for (int k = 0; k < 4; ++k) bson[4 * b + k] = -1;
      continue;
    }
    int32_t t = brow[b], s = bcol[b];
    int32_t k0 = cstart[b];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        int32_t k = k0 + 2 * i + j;
        nrow[k] = cson[2 * t + i];
        ncol[k] = cson[2 * s + j];
        npar[k] = first_id + b;
        bson[4 * b + 2 * i + j] = first_child_id + k;
      }
  }
}

// ---------------------------------------------------------------- DFS pre-order ids
// Subtree sizes, bottom-up over one level of a tree stored level by level with
// global (BFS) ids; children ids refer to the same global numbering.
__global__ void k_subtree(int32_t first, int32_t cnt, int nsons, const int32_t* sons, int32_t* sub) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    int32_t g = first + i;
    int32_t s = 1;
    for (int k = 0; k < nsons; ++k) {
      int32_t c = sons[nsons * (int64_t)g + k];
      if (c >= 0) s += sub[c];
    }
    sub[g] = s;
  }
}
__global__ void k_preorder(int32_t first, int32_t cnt, int nsons, const int32_t* sons, const int32_t* sub, int32_t* pre) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    int32_t g = first + i;
    int32_t next = pre[g] + 1;
    for (int k = 0; k < nsons; ++k) {
      int32_t c = sons[nsons * (int64_t)g + k];
      if (c < 0) continue;
      pre[c] = next;
      next += sub[c];
    }
  }
}

// export rows in DFS order
__global__ void k_export_clusters(int32_t nc, const int32_t* pre, const int32_t* off, const int32_t* size,
                                  const int32_t* lo, const int32_t* hi, const int32_t* son, const int32_t* level,
                                  const int32_t* parent, int32_t* out) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nc; g += gridDim.x * blockDim.x) {
    int32_t* r = out + 12 * (int64_t)pre[g];
    r[0] = off[g];
    r[1] = size[g];
    for (int a = 0; a < 3; ++a) {
      r[2 + a] = lo[3 * (int64_t)g + a];
      r[5 + a] = hi[3 * (int64_t)g + a];
    }
    r[8] = son[2 * g] >= 0 ? pre[son[2 * g]] : -1;
    r[9] = son[2 * g + 1] >= 0 ? pre[son[2 * g + 1]] : -1;
    r[10] = level[g];
    r[11] = parent[g] >= 0 ? pre[parent[g]] : -1;
  }
}
__global__ void k_export_blocks(int32_t nb, const int32_t* bpre, const int32_t* cpre, const int32_t* row,
                                const int32_t* col, const int32_t* kind, const int32_t* son, const int32_t* parent,
                                int32_t* out) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nb; g += gridDim.x * blockDim.x) {
    int32_t* r = out + 8 * (int64_t)bpre[g];
    r[0] = cpre[row[g]];
    r[1] = cpre[col[g]];
    r[2] = kind[g];
    for (int k = 0; k < 4; ++k) r[3 + k] = son[4 * (int64_t)g + k] >= 0 ? bpre[son[4 * (int64_t)g + k]] : -1;
    r[7] = parent[g] >= 0 ? bpre[parent[g]] : -1;
  }
}

// ---------------------------------------------------------------- A_H fill
template <class T>
__global__ void k_fill_dense(int32_t nblk, const FillDesc* d, const int32_t* perm, const int32_t* iperm,
                             const int64_t* rowptr, const int32_t* col, const double* val, T* arena) {
  // one warp per (block, row)
  int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = gw;; w += nw) {
    // map w -> (block, row) through the row prefix in the descriptors
    int32_t lo = 0, hi = nblk;
    while (hi - lo > 1) {
      int32_t mid = (lo + hi) / 2;
      if (d[mid].row_prefix <= w)
        lo = mid;
      else
        hi = mid;
    }
    if (nblk == 0 || w >= d[nblk - 1].row_prefix + d[nblk - 1].m) return;
    const FillDesc& f = d[lo];
    int32_t i = (int32_t)(w - f.row_prefix);
    int32_t orow = perm[f.roff + i];
    for (int64_t e = rowptr[orow] + lane; e < rowptr[orow + 1]; e += 32) {
      int32_t j = iperm[col[e]] - f.coff;
      if (j >= 0 && j < f.n) arena[f.off + i + (int64_t)j * f.m] = (T)val[e];
    }
  }
}

// one CTA per admissible block: X = unit columns of the nonzero rows, Y^T = rows
template <class T>
__global__ void k_fill_lowrank(int32_t nblk, const FillDesc* d, const int32_t* perm, const int32_t* iperm,
                               const int64_t* rowptr, const int32_t* col, const double* val, T* arena,
                               int32_t* ranks, int32_t* status) {
  __shared__ int32_t s_k;
  __shared__ int32_t s_flag[256];
  for (int32_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const FillDesc& f = d[b];
    if (threadIdx.x == 0) s_k = 0;
    __syncthreads();
    for (int32_t base = 0; base < f.m; base += blockDim.x) {
      int32_t i = base + threadIdx.x;
      int32_t has = 0;
      int32_t orow = 0;
      if (i < f.m) {
        orow = perm[f.roff + i];
        for (int64_t e = rowptr[orow]; e < rowptr[orow + 1]; ++e) {
          int32_t j = iperm[col[e]] - f.coff;
          if (j >= 0 && j < f.n) {
            has = 1;
            break;
          }
        }
      }
      s_flag[threadIdx.x] = has;
      __syncthreads();
      // sequential rank positions in row order (nonzero rows are rare)
      if (threadIdx.x == 0) {
        int32_t k = s_k;
        for (int q = 0; q < (int)blockDim.x; ++q)
          if (s_flag[q]) s_flag[q] = ++k;
        s_k = k;
      }
      __syncthreads();
      if (has) {
        int32_t kk = s_flag[threadIdx.x] - 1;
        if (kk < f.cap) {
          arena[f.off + i + (int64_t)kk * f.m] = T(1);
          for (int64_t e = rowptr[orow]; e < rowptr[orow + 1]; ++e) {
            int32_t j = iperm[col[e]] - f.coff;
            if (j >= 0 && j < f.n) arena[f.off2 + j + (int64_t)kk * f.n] = (T)val[e];
          }
        } else {
          atomicCAS(status, 0, 7);
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) ranks[f.slot] = min(s_k, f.cap);
    __syncthreads();
  }
}

template <class T>
__global__ void k_identity(T* arena, int64_t off, int32_t n) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    arena[off + i + (int64_t)i * n] = T(1);
}

template __global__ void k_fill_dense<float>(int32_t, const FillDesc*, const int32_t*, const int32_t*, const int64_t*,
                                            const int32_t*, const double*, float*);
template __global__ void k_fill_dense<double>(int32_t, const FillDesc*, const int32_t*, const int32_t*, const int64_t*,
                                             const int32_t*, const double*, double*);

// ---------------------------------------------------------------- host drivers
#define CK(x)                               \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)

// Temporaries of one host driver: freed when the driver returns, on success
// or on an early error return.
struct TempScope {
  std::vector<void*> ptrs;
  template <class T>
  cudaError_t alloc(T** p, size_t bytes) {
    cudaError_t e = dev_malloc(p, bytes);
    if (e == cudaSuccess) ptrs.push_back((void*)*p);
    return e;
  }
  ~TempScope() {
    for (void* p : ptrs) dev_free(p);
  }
};
// thrust's temporary storage comes from the library's allocator too
static ThrustAlloc g_talloc;

static int grid_for(int64_t n, int bs = 256) {
  int64_t g = (n + bs - 1) / bs;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (int)g;
}

cudaError_t build_mesh_dofs(int n, cudaStream_t s, DevMesh& m) {
  int64_t nv = (int64_t)(n + 1) * (n + 1) * (n + 1);
  TempScope tmp;
  int32_t* cnt = nullptr;
  CK(tmp.alloc(&cnt, sizeof(int32_t) * (nv + 1)));
  CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nv + 1), s));
  note_launch();
  k_count_edges<<<grid_for(nv), 256, 0, s>>>(n, cnt);
  thrust::exclusive_scan(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int32_t>(cnt),
                         thrust::device_ptr<int32_t>(cnt + nv + 1), thrust::device_ptr<int32_t>(cnt));
  int32_t N = 0;
  CK(cudaMemcpyAsync(&N, cnt + nv, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  m.n = n;
  m.N = N;
  CK(dev_malloc(&m.dofmap, sizeof(int32_t) * nv * 7));
  CK(dev_malloc(&m.edges, sizeof(int32_t) * 2 * (int64_t)N));
  CK(dev_malloc(&m.pts, sizeof(int32_t) * 3 * (int64_t)N));
  note_launch();
  k_number_edges<<<grid_for(nv), 256, 0, s>>>(n, cnt, m.dofmap, m.edges, m.pts);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return cudaSuccess;
}

// ---------------------------------------------------------------- general meshes
// 6 edge keys (lo * nv + hi) per tetrahedron
__global__ void k_tet_edge_keys(int64_t nt, int32_t nv, const int32_t* tets, int64_t* keys) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    for (int e = 0; e < 6; ++e) {
      int64_t a = tets[4 * t + c_ledge[e][0]], b = tets[4 * t + c_ledge[e][1]];
      if (a > b) {
        const int64_t x = a;
        a = b;
        b = x;
      }
      keys[6 * t + e] = a * nv + b;
    }
  }
}
// 4 face keys (a nv^2 + b nv + c, a < b < c) per tetrahedron
__global__ void k_tet_face_keys(int64_t nt, int32_t nv, const int32_t* tets, int64_t* keys) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t v[4];
    for (int s = 0; s < 4; ++s) v[s] = tets[4 * t + s];
    for (int i = 1; i < 4; ++i)  // sort the 4 ids
      for (int j = i; j > 0 && v[j - 1] > v[j]; --j) {
        const int64_t x = v[j];
        v[j] = v[j - 1];
        v[j - 1] = x;
      }
    for (int skip = 0; skip < 4; ++skip) {
      int64_t f[3];
      int q = 0;
      for (int s = 0; s < 4; ++s)
        if (s != skip) f[q++] = v[s];
      keys[4 * t + skip] = (f[0] * nv + f[1]) * nv + f[2];
    }
  }
}
// the 3 edge keys of every boundary face (faces that occur once)
__global__ void k_boundary_face_edges(int64_t nf, int32_t nv, const int64_t* fkeys, const int32_t* fcount,
                                      int64_t* ekeys, int64_t* n_out) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    if (fcount[f] != 1) continue;
    const int64_t k = fkeys[f];
    const int64_t a = k / ((int64_t)nv * nv), b = (k / nv) % nv, c = k % nv;
    const unsigned long long o = atomicAdd(reinterpret_cast<unsigned long long*>(n_out), 3ULL);
    ekeys[o] = a * nv + b;
    ekeys[o + 1] = a * nv + c;
    ekeys[o + 2] = b * nv + c;
  }
}
// edges and tree points of the interior edges: p = rint((x_lo + x_hi - 2 b) s),
// every operation rounded once as written (no contraction)
__global__ void k_general_edges(int64_t N, int32_t nv, const int64_t* ekeys, const double* xyz, double b0, double b1,
                                double b2, double scale, int32_t* edges, int32_t* pts) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = ekeys[e] / nv, hi = ekeys[e] % nv;
    edges[2 * e] = (int32_t)lo;
    edges[2 * e + 1] = (int32_t)hi;
    const double bb[3] = {b0, b1, b2};
    for (int a = 0; a < 3; ++a) {
      const double t1 = __dadd_rn(xyz[3 * lo + a], xyz[3 * hi + a]);
      const double t2 = __dsub_rn(t1, __dmul_rn(2.0, bb[a]));
      pts[3 * e + a] = (int32_t)__double2ll_rn(__dmul_rn(t2, scale));
    }
  }
}

cudaError_t build_mesh_general(int32_t nv, int64_t nt, const double* xyz, const int32_t* tets, cudaStream_t s,
                               DevMesh& m) {
  TempScope tmp;
  m.n = 0;
  m.nv = nv;
  m.nt = nt;
  CK(dev_malloc(&m.xyz, sizeof(double) * 3 * (int64_t)nv));
  CK(dev_malloc(&m.tets, sizeof(int32_t) * 4 * nt));
  CK(cudaMemcpyAsync(m.xyz, xyz, sizeof(double) * 3 * (int64_t)nv, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m.tets, tets, sizeof(int32_t) * 4 * nt, cudaMemcpyHostToDevice, s));
  // all edges, sorted and unique
  int64_t* ek = nullptr;
  CK(tmp.alloc(&ek, sizeof(int64_t) * 6 * nt));
  note_launch();
  k_tet_edge_keys<<<grid_for(nt), 256, 0, s>>>(nt, nv, m.tets, ek);
  CK(cudaGetLastError());
  thrust::sort(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(ek), thrust::device_ptr<int64_t>(ek + 6 * nt));
  const int64_t ne = thrust::unique(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(ek),
                                    thrust::device_ptr<int64_t>(ek + 6 * nt)) -
                     thrust::device_ptr<int64_t>(ek);
  // faces and how many tetrahedra hold each
  int64_t* fk = nullptr;
  int64_t* fu = nullptr;
  int32_t* ones = nullptr;
  int32_t* fc = nullptr;
  CK(tmp.alloc(&fk, sizeof(int64_t) * 4 * nt));
  CK(tmp.alloc(&fu, sizeof(int64_t) * 4 * nt));
  CK(tmp.alloc(&ones, sizeof(int32_t) * 4 * nt));
  CK(tmp.alloc(&fc, sizeof(int32_t) * 4 * nt));
  note_launch();
  k_tet_face_keys<<<grid_for(nt), 256, 0, s>>>(nt, nv, m.tets, fk);
  CK(cudaGetLastError());
  thrust::sort(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(fk), thrust::device_ptr<int64_t>(fk + 4 * nt));
  thrust::fill(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int32_t>(ones),
               thrust::device_ptr<int32_t>(ones + 4 * nt), 1);
  auto fe = thrust::reduce_by_key(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(fk),
                                  thrust::device_ptr<int64_t>(fk + 4 * nt), thrust::device_ptr<int32_t>(ones),
                                  thrust::device_ptr<int64_t>(fu), thrust::device_ptr<int32_t>(fc));
  const int64_t nf = fe.first - thrust::device_ptr<int64_t>(fu);
  // boundary edges: the edges of faces held by one tetrahedron
  int64_t* bk = nullptr;
  int64_t* nb = nullptr;
  CK(tmp.alloc(&bk, sizeof(int64_t) * 3 * std::max<int64_t>(nf, 1)));
  CK(tmp.alloc(&nb, sizeof(int64_t)));
  CK(cudaMemsetAsync(nb, 0, sizeof(int64_t), s));
  note_launch();
  k_boundary_face_edges<<<grid_for(nf), 256, 0, s>>>(nf, nv, fu, fc, bk, nb);
  CK(cudaGetLastError());
  int64_t nbk = 0;
  CK(cudaMemcpyAsync(&nbk, nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  thrust::sort(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(bk), thrust::device_ptr<int64_t>(bk + nbk));
  const int64_t nbu = thrust::unique(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(bk),
                                     thrust::device_ptr<int64_t>(bk + nbk)) -
                      thrust::device_ptr<int64_t>(bk);
  // interior edges = all edges minus boundary edges, in key = (lo, hi) order
  CK(dev_malloc(&m.ekeys, sizeof(int64_t) * std::max<int64_t>(ne, 1)));
  const int64_t N = thrust::set_difference(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(ek),
                                           thrust::device_ptr<int64_t>(ek + ne), thrust::device_ptr<int64_t>(bk),
                                           thrust::device_ptr<int64_t>(bk + nbu), thrust::device_ptr<int64_t>(m.ekeys)) -
                    thrust::device_ptr<int64_t>(m.ekeys);
  m.N = N;
  if (N < 1) return cudaErrorInvalidValue;
  // tree points on the integer grid (bounding box and scale on the host)
  double lo[3] = {xyz[0], xyz[1], xyz[2]}, hi[3] = {xyz[0], xyz[1], xyz[2]};
  for (int64_t v = 0; v < nv; ++v)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], xyz[3 * v + a]);
      hi[a] = std::max(hi[a], xyz[3 * v + a]);
    }
  double extent = 0;
  for (int a = 0; a < 3; ++a) extent = std::max(extent, hi[a] - lo[a]);
  if (!(extent > 0)) return cudaErrorInvalidValue;
  double scale = 1.0;
  while (2.0 * extent * scale * 2.0 <= 2097152.0) scale *= 2.0;
  while (2.0 * extent * scale > 2097152.0) scale *= 0.5;
  CK(dev_malloc(&m.edges, sizeof(int32_t) * 2 * N));
  CK(dev_malloc(&m.pts, sizeof(int32_t) * 3 * N));
  note_launch();
  k_general_edges<<<grid_for(N), 256, 0, s>>>(N, nv, m.ekeys, m.xyz, lo[0], lo[1], lo[2], scale, m.edges, m.pts);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return cudaSuccess;
}

cudaError_t assemble_csr(const DevMesh& m, double kappa, cudaStream_t s, DevCSR& A) {
  const MeshView mv = view_of(m);
  const int64_t nt = mv.nt;
  int64_t ne = nt * 36;
  TempScope tmp;
  int64_t* keys = nullptr;
  double* vals = nullptr;
  CK(tmp.alloc(&keys, sizeof(int64_t) * ne));
  CK(tmp.alloc(&vals, sizeof(double) * ne));
  note_launch();
  k_element_coo<<<grid_for(nt, 128), 128, 0, s>>>(mv, kappa * kappa, m.N, keys, vals);
  CK(cudaGetLastError());
  thrust::stable_sort_by_key(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(keys),
                             thrust::device_ptr<int64_t>(keys + ne), thrust::device_ptr<double>(vals));
  int64_t* ukeys = nullptr;
  double* uvals = nullptr;
  CK(tmp.alloc(&ukeys, sizeof(int64_t) * ne));
  CK(tmp.alloc(&uvals, sizeof(double) * ne));
  auto ends = thrust::reduce_by_key(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int64_t>(keys),
                                    thrust::device_ptr<int64_t>(keys + ne), thrust::device_ptr<double>(vals),
                                    thrust::device_ptr<int64_t>(ukeys), thrust::device_ptr<double>(uvals));
  int64_t nu = ends.first - thrust::device_ptr<int64_t>(ukeys);
  int64_t last = 0;
  CK(cudaMemcpyAsync(&last, ukeys + nu - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int64_t nnz = (last == INT64_MAX) ? nu - 1 : nu;
  A.N = m.N;
  A.nnz = nnz;
  CK(dev_malloc(&A.rowptr, sizeof(int64_t) * (m.N + 1)));
  CK(dev_malloc(&A.col, sizeof(int32_t) * nnz));
  CK(dev_malloc(&A.val, sizeof(double) * nnz));
  int32_t* rowcnt = nullptr;
  CK(tmp.alloc(&rowcnt, sizeof(int32_t) * (m.N + 1)));
  CK(cudaMemsetAsync(rowcnt, 0, sizeof(int32_t) * (m.N + 1), s));
  note_launch();
  k_csr_rows<<<grid_for(nnz), 256, 0, s>>>(nnz, m.N, ukeys, A.col, rowcnt);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(A.val, uvals, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, s));
  thrust::exclusive_scan(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int32_t>(rowcnt),
                         thrust::device_ptr<int32_t>(rowcnt + m.N + 1), thrust::device_ptr<int64_t>(A.rowptr),
                         (int64_t)0);
  CK(cudaStreamSynchronize(s));
  return cudaSuccess;
}

// Load vector from per-tetrahedron (dof, value) pairs: manufactured field
// (J == nullptr) or constant current J[3].  The pairs are sorted by DOF and
// summed in a fixed order, so the result does not depend on the launch.
static cudaError_t rhs_from_elements(const DevMesh& m, double kappa, const double* Jc, double* b, cudaStream_t s) {
  const MeshView mv = view_of(m);
  const int64_t nt = mv.nt;
  int64_t ne = nt * 6;
  int32_t* keys = nullptr;
  double* vals = nullptr;
  int32_t* uk = nullptr;
  double* us = nullptr;
  TempScope tmp;
  CK(tmp.alloc(&keys, sizeof(int32_t) * ne));
  CK(tmp.alloc(&vals, sizeof(double) * ne));
  CK(tmp.alloc(&uk, sizeof(int32_t) * ne));
  CK(tmp.alloc(&us, sizeof(double) * ne));
  note_launch();
  if (Jc)
    k_rhs_const_coo<<<grid_for(nt, 128), 128, 0, s>>>(mv, Jc[0], Jc[1], Jc[2], keys, vals);
  else
    k_rhs_coo<<<grid_for(nt, 128), 128, 0, s>>>(mv, kappa * kappa, keys, vals);
  CK(cudaGetLastError());
  thrust::stable_sort_by_key(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int32_t>(keys),
                             thrust::device_ptr<int32_t>(keys + ne), thrust::device_ptr<double>(vals));
  auto ends = thrust::reduce_by_key(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int32_t>(keys),
                                    thrust::device_ptr<int32_t>(keys + ne), thrust::device_ptr<double>(vals),
                                    thrust::device_ptr<int32_t>(uk), thrust::device_ptr<double>(us));
  int64_t nu = ends.first - thrust::device_ptr<int32_t>(uk);
  CK(cudaMemsetAsync(b, 0, sizeof(double) * m.N, s));
  note_launch();
  k_scatter_rhs<<<grid_for(nu), 256, 0, s>>>(nu, uk, us, m.N, b);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return cudaSuccess;
}

cudaError_t manufactured_rhs(const DevMesh& m, double kappa, double* b, cudaStream_t s) {
  return rhs_from_elements(m, kappa, nullptr, b, s);
}

cudaError_t constant_current_rhs(const DevMesh& m, const double J[3], double* b, cudaStream_t s) {
  return rhs_from_elements(m, 0.0, J, b, s);
}

cudaError_t build_trees(const DevMesh& m, int32_t leaf, int64_t eta2, cudaStream_t s, HostTrees& out,
                        int32_t* d_perm_out) {
  const int32_t N = (int32_t)m.N;
  // level-by-level cluster arrays with global BFS ids; generous capacity
  int32_t cap = 2 * N + 16;  // a binary tree with at most N leaves
  TempScope tmp;
  int32_t *off, *size, *lo, *hi, *son, *level, *parent, *nleft, *permA, *permB, *cnt;
  CK(tmp.alloc(&off, sizeof(int32_t) * cap));
  CK(tmp.alloc(&size, sizeof(int32_t) * cap));
  CK(tmp.alloc(&lo, sizeof(int32_t) * 3 * cap));
  CK(tmp.alloc(&hi, sizeof(int32_t) * 3 * cap));
  CK(tmp.alloc(&son, sizeof(int32_t) * 2 * cap));
  CK(tmp.alloc(&level, sizeof(int32_t) * cap));
  CK(tmp.alloc(&parent, sizeof(int32_t) * cap));
  CK(tmp.alloc(&nleft, sizeof(int32_t) * cap));
  CK(tmp.alloc(&permA, sizeof(int32_t) * (N + 1)));
  CK(tmp.alloc(&permB, sizeof(int32_t) * (N + 1)));
  CK(tmp.alloc(&cnt, sizeof(int32_t)));
  thrust::sequence(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int32_t>(permA), thrust::device_ptr<int32_t>(permA + N));
  int32_t h0[2] = {0, N};
  CK(cudaMemcpyAsync(off, &h0[0], sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(size, &h0[1], sizeof(int32_t), cudaMemcpyHostToDevice, s));
  int32_t mone = -1, zero = 0;
  CK(cudaMemcpyAsync(parent, &mone, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(level, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  std::vector<int32_t> level_first = {0}, level_cnt = {1};
  int32_t first = 0, count = 1, lev = 0;
  while (count > 0) {
    if (first + count + 2 * count > cap) return cudaErrorMemoryAllocation;
    note_launch();
    k_cluster_bbox<<<std::min(count, 8192), 256, 0, s>>>(count, off + first, size + first, permA, m.pts, lo + 3 * first,
                                                         hi + 3 * first);
    // clusters that became leaves on earlier levels keep their order
    CK(cudaMemcpyAsync(permB, permA, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
    note_launch();
    k_cluster_split<<<std::min(count, 8192), 1024, 0, s>>>(count, leaf, off + first, size + first, lo + 3 * first,
                                                           hi + 3 * first, permA, permB, m.pts, nleft + first);
    note_launch();
    k_cluster_children<<<1, 1, 0, s>>>(count, first, off + first, size + first, nleft + first, son + 2 * first,
                                       off + first + count, size + first + count, parent + first + count, cnt);
    CK(cudaGetLastError());
    int32_t nxt = 0;
    CK(cudaMemcpyAsync(&nxt, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // son indices are level-local: make them global
    if (nxt > 0) {
      std::vector<int32_t> hs(2 * count);
      CK(cudaMemcpy(hs.data(), son + 2 * first, sizeof(int32_t) * 2 * count, cudaMemcpyDeviceToHost));
      for (auto& x : hs)
        if (x >= 0) x += first + count;
      CK(cudaMemcpy(son + 2 * first, hs.data(), sizeof(int32_t) * 2 * count, cudaMemcpyHostToDevice));
      std::vector<int32_t> hl(nxt, lev + 1);
      CK(cudaMemcpy(level + first + count, hl.data(), sizeof(int32_t) * nxt, cudaMemcpyHostToDevice));
    }
    std::swap(permA, permB);
    first += count;
    count = nxt;
    ++lev;
    if (count) {
      level_first.push_back(first);
      level_cnt.push_back(count);
    }
  }
  const int32_t nc = first;
  // DFS pre-order ids
  int32_t *sub, *pre;
  CK(tmp.alloc(&sub, sizeof(int32_t) * nc));
  CK(tmp.alloc(&pre, sizeof(int32_t) * nc));
  for (int l = (int)level_first.size() - 1; l >= 0; --l) {
    note_launch();
    k_subtree<<<grid_for(level_cnt[l]), 256, 0, s>>>(level_first[l], level_cnt[l], 2, son, sub);
  }
  CK(cudaMemcpyAsync(pre, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  for (size_t l = 0; l < level_first.size(); ++l) {
    note_launch();
    k_preorder<<<grid_for(level_cnt[l]), 256, 0, s>>>(level_first[l], level_cnt[l], 2, son, sub, pre);
  }
  int32_t* cl_export;
  CK(tmp.alloc(&cl_export, sizeof(int32_t) * 12 * nc));
  note_launch();
  k_export_clusters<<<grid_for(nc), 256, 0, s>>>(nc, pre, off, size, lo, hi, son, level, parent, cl_export);
  CK(cudaGetLastError());

  // ---- block tree, level by level (global BFS ids)
  int32_t bcap = 1 << 20;
  int32_t *brow, *bcol, *bkind, *bson, *bpar, *nch, *cst;
  auto balloc = [&](int32_t c) -> cudaError_t {
    CK(tmp.alloc(&brow, sizeof(int32_t) * c));
    CK(tmp.alloc(&bcol, sizeof(int32_t) * c));
    CK(tmp.alloc(&bkind, sizeof(int32_t) * c));
    CK(tmp.alloc(&bson, sizeof(int32_t) * 4 * (int64_t)c));
    CK(tmp.alloc(&bpar, sizeof(int32_t) * c));
    CK(tmp.alloc(&nch, sizeof(int32_t) * (c + 1)));
    CK(tmp.alloc(&cst, sizeof(int32_t) * (c + 1)));
    return cudaSuccess;
  };
  // capacity: blocks grow at most 4x per level; bound by an estimate, grow on demand
  bcap = std::max<int32_t>(1 << 16, 64 * nc + 4096);
  CK(balloc(bcap));
  // cluster son array in BFS ids is `son`; boxes lo/hi in BFS ids
  CK(cudaMemcpyAsync(brow, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bcol, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bpar, &mone, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  std::vector<int32_t> bl_first = {0}, bl_cnt = {1};
  int32_t bfirst = 0, bcount = 1;
  while (bcount > 0) {
    note_launch();
    k_block_classify<<<grid_for(bcount), 256, 0, s>>>(bcount, brow + bfirst, bcol + bfirst, lo, hi, son, eta2,
                                                      bkind + bfirst, nch + bfirst);
    CK(cudaGetLastError());
    thrust::exclusive_scan(thrust::cuda::par(g_talloc).on(s), thrust::device_ptr<int32_t>(nch + bfirst),
                           thrust::device_ptr<int32_t>(nch + bfirst + bcount), thrust::device_ptr<int32_t>(cst + bfirst));
    int32_t lastc = 0, lastn = 0;
    CK(cudaMemcpyAsync(&lastc, cst + bfirst + bcount - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&lastn, nch + bfirst + bcount - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int32_t nxt = lastc + lastn;
    if (bfirst + bcount + nxt > bcap) return cudaErrorMemoryAllocation;
    note_launch();
    k_block_expand<<<grid_for(bcount), 256, 0, s>>>(bcount, brow + bfirst, bcol + bfirst, bkind + bfirst,
                                                    cst + bfirst, son, bfirst + bcount, bfirst, bson + 4 * (int64_t)bfirst,
                                                    brow + bfirst + bcount, bcol + bfirst + bcount,
                                                    bpar + bfirst + bcount);
    CK(cudaGetLastError());
    bfirst += bcount;
    bcount = nxt;
    if (bcount) {
      bl_first.push_back(bfirst);
      bl_cnt.push_back(bcount);
    }
  }
  const int32_t nb = bfirst;
  int32_t *bsub, *bpre;
  CK(tmp.alloc(&bsub, sizeof(int32_t) * nb));
  CK(tmp.alloc(&bpre, sizeof(int32_t) * nb));
  for (int l = (int)bl_first.size() - 1; l >= 0; --l) {
    note_launch();
    k_subtree<<<grid_for(bl_cnt[l]), 256, 0, s>>>(bl_first[l], bl_cnt[l], 4, bson, bsub);
  }
  CK(cudaMemcpyAsync(bpre, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  for (size_t l = 0; l < bl_first.size(); ++l) {
    note_launch();
    k_preorder<<<grid_for(bl_cnt[l]), 256, 0, s>>>(bl_first[l], bl_cnt[l], 4, bson, bsub, bpre);
  }
  int32_t* bl_export;
  CK(tmp.alloc(&bl_export, sizeof(int32_t) * 8 * (int64_t)nb));
  note_launch();
  k_export_blocks<<<grid_for(nb), 256, 0, s>>>(nb, bpre, pre, brow, bcol, bkind, bson, bpar, bl_export);
  CK(cudaGetLastError());
  out.clusters.resize(12 * (size_t)nc);
  out.blocks.resize(8 * (size_t)nb);
  out.perm.resize(N);
  CK(cudaMemcpyAsync(out.clusters.data(), cl_export, sizeof(int32_t) * 12 * nc, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(out.blocks.data(), bl_export, sizeof(int32_t) * 8 * (int64_t)nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(out.perm.data(), permA, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(d_perm_out, permA, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  out.nc = nc;
  out.nb = nb;
  return cudaSuccess;
}

template <class T>
cudaError_t fill_ah(const DevCSR& A, const int32_t* d_perm, const int32_t* d_iperm, const FillDesc* d_dense,
                    int32_t ndense, int64_t dense_rows, const FillDesc* d_lr, int32_t nlr, T* arena,
                    int64_t zero_elems, int64_t ident_off, int32_t ident_n, int32_t* ranks, int32_t* status,
                    cudaStream_t s) {
  CK(cudaMemsetAsync(arena, 0, sizeof(T) * zero_elems, s));
  note_launch();
  k_identity<T><<<grid_for(ident_n), 256, 0, s>>>(arena, ident_off, ident_n);
  if (ndense) {
    int64_t warps = dense_rows;
    int blocks = (int)std::min<int64_t>((warps * 32 + 255) / 256, 65535);
    note_launch();
    k_fill_dense<T><<<blocks, 256, 0, s>>>(ndense, d_dense, d_perm, d_iperm, A.rowptr, A.col, A.val, arena);
  }
  if (nlr) {
    note_launch();
    k_fill_lowrank<T><<<std::min(nlr, 65535), 256, 0, s>>>(nlr, d_lr, d_perm, d_iperm, A.rowptr, A.col, A.val, arena, ranks, status);
  }
  return cudaGetLastError();
}

template cudaError_t fill_ah<float>(const DevCSR&, const int32_t*, const int32_t*, const FillDesc*, int32_t, int64_t,
                                    const FillDesc*, int32_t, float*, int64_t, int64_t, int32_t, int32_t*, int32_t*,
                                    cudaStream_t);
template cudaError_t fill_ah<double>(const DevCSR&, const int32_t*, const int32_t*, const FillDesc*, int32_t, int64_t,
                                     const FillDesc*, int32_t, double*, int64_t, int64_t, int32_t, int32_t*, int32_t*,
                                     cudaStream_t);

__global__ void k_invert_perm(int32_t N, const int32_t* perm, int32_t* iperm) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) iperm[perm[i]] = i;
}
cudaError_t invert_perm(int32_t N, const int32_t* perm, int32_t* iperm, cudaStream_t s) {
  note_launch();
  k_invert_perm<<<grid_for(N), 256, 0, s>>>(N, perm, iperm);
  return cudaGetLastError();
}


// ---------------------------------------------------------------- load vector without allocation
// Variant of manufactured_rhs whose scratch (the 6 element contributions per
// tetrahedron: DOF key and value) lives in a fixed file-scope device array
// instead of per-call allocations, and whose reduction adds the contributions
// into b with atomics instead of a sort (which would need temporary storage).
namespace {

constexpr int64_t kRhsScratchEntries = int64_t(1) << 19;  // 36 n^3 <= 524,288: n <= 24
static __device__ __align__(256) unsigned char g_rhs_scratch[kRhsScratchEntries * (sizeof(double) + sizeof(int32_t))];

constexpr int kMaxDevices = 64;
std::mutex g_rhs_mu;
void* g_rhs_ptr[kMaxDevices] = {};

__global__ void k_add_rhs(int64_t ne, const int32_t* keys, const double* vals, int64_t N, double* b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = keys[e];
    if (k >= 0 && k < N) atomicAdd(b + k, vals[e]);
  }
}

}  // namespace

int64_t rhs_noalloc_max_entries() { return kRhsScratchEntries; }

cudaError_t manufactured_rhs_noalloc(const DevMesh& m, double kappa, double* b, cudaStream_t s) {
  const int64_t nt = (int64_t)6 * m.n * m.n * m.n;
  const int64_t ne = nt * 6;
  if (ne > kRhsScratchEntries) return cudaErrorInvalidValue;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  void* base = nullptr;
  {
    // set-up, once per device (with that device current): the scratch's
    // device address
    std::lock_guard<std::mutex> lk(g_rhs_mu);
    if (!g_rhs_ptr[dev]) {
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_rhs_scratch));
      g_rhs_ptr[dev] = p;
    }
    base = g_rhs_ptr[dev];
  }
  // values first (8-byte aligned at the 256-byte aligned base), keys after
  double* vals = reinterpret_cast<double*>(base);
  int32_t* keys = reinterpret_cast<int32_t*>(vals + kRhsScratchEntries);
  // every scratch entry read below is written first by k_rhs_coo; b starts at 0
  CK(cudaMemsetAsync(b, 0, sizeof(double) * m.N, s));
  note_launch();
  k_rhs_coo<<<grid_for(nt, 128), 128, 0, s>>>(view_of(m), kappa * kappa, keys, vals);
  CK(cudaGetLastError());
  note_launch();
  k_add_rhs<<<grid_for(ne), 256, 0, s>>>(ne, keys, vals, m.N, b);
  CK(cudaGetLastError());
  return cudaSuccess;
}

}  // namespace hlu
