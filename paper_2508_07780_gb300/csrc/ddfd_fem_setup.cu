// Host set-up of the element-by-element FEM rows: the explicit P1 mesh of
// the FEM cube (the Kuhn split, fem_kind = DDFD_FEM_EBE, or a locally refined
// mesh, fem_kind = DDFD_FEM_MESH), its per-tet gradients, row incidences and
// lumped masses, packed into shared-memory blocks for the gather kernel
// (ddfd_ebe.cu) and uploaded.
#include "ddfd_host.h"

using namespace ddfd;
using namespace ddfd::host;

namespace {

// Explicit P1 mesh of the FEM cube for the element-by-element path: the six
// Kuhn tetrahedra of every cube of [a, b]^3 as a tet list with per-tet
// sqrt|K| g (from the inverse of [1 x] in FP64), the incidences of the nodes
// strictly inside the cube (the rows the FEM updates) and their lumped masses.
// Packs the element-by-element rows into shared-memory blocks and uploads
// them with the rows' node offsets and mass scales (both mesh kinds).
int upload_ebe(ddfd_problem *p, long long rows, long long ntet, const std::vector<int> &tnode,
               const std::vector<double> &tgrad, const std::vector<int> &rptr, const std::vector<int> &itet,
               const std::vector<int> &iloc, const std::vector<int> &rnode, const std::vector<double> &scale,
               const std::vector<double> &rpos, const std::vector<unsigned char> *stencil = nullptr) {
  // rows marked in *stencil take the Kuhn block stencil; the others are gathered
  std::vector<unsigned char> use;
  std::vector<int> klist;
  if (stencil) {
    use.assign((size_t)rows, 1);
    for (size_t r = 0; r < stencil->size(); ++r)
      if ((*stencil)[r]) {
        use[r] = 0;
        klist.push_back((int)r);
      }
  }
  {
    // algorithmic bytes: the tets incident to gathered rows and their nodes, once each
    std::vector<unsigned char> tmark((size_t)ntet, 0);
    long long grows = 0, nt_used = 0;
    for (long long r = 0; r < rows; ++r) {
      if (stencil && !use[r]) continue;
      ++grows;
      for (int q = rptr[r]; q < rptr[r + 1]; ++q) tmark[itet[q]] = 1;
    }
    std::vector<int> nodes;
    for (long long t = 0; t < ntet; ++t)
      if (tmark[t]) {
        ++nt_used;
        for (int q = 0; q < 4; ++q) nodes.push_back(tnode[t * 4 + q]);
      }
    std::sort(nodes.begin(), nodes.end());
    const long long nn_used = std::unique(nodes.begin(), nodes.end()) - nodes.begin();
    const long long es = (long long)p->esz, kr = (long long)klist.size();
    p->ebe_bytes_fwd = nt_used * (16 + 12 * es) + nn_used * 4 * es + grows * 3 * es + kr * 7 * es;
    p->ebe_bytes_adj = nt_used * (16 + 12 * es) + nn_used * 3 * es + grows * 6 * es + kr * 10 * es;
  }
  EbePack pk;
  std::string m;
  if (!pack_ebe_blocks(rows, ntet, tnode.data(), tgrad.data(), rptr.data(), itet.data(), iloc.data(), rpos.data(),
                       (int)p->esz, &pk, &m, stencil ? use.data() : nullptr))
    return fail(p, DDFD_E_ARG, m);
  if (!klist.empty()) {
    int st;
    if ((st = dalloc_t(p, klist.size(), &p->kuhn_list))) return st;
    CK(cudaMemcpy(p->kuhn_list, klist.data(), klist.size() * sizeof(int), cudaMemcpyHostToDevice));
    p->kuhn_n = (int)klist.size();
  }
  int st;
  const size_t es = p->esz;
  if ((st = dalloc_t(p, (size_t)rows, &p->ebe_row_node)) || (st = dalloc_t(p, (size_t)rows, &p->ebe_scale)) ||
      (st = dalloc_t(p, pk.blocks.size(), &p->ebe_blocks)) || (st = dalloc_t(p, pk.blob.size(), &p->ebe_blob)) ||
      (st = dalloc_t(p, pk.nodes.size(), &p->ebe_blk_nodes)) || (st = dalloc_t(p, pk.rows.size(), &p->ebe_blk_rows)) ||
      (st = dalloc(p, 3 * (size_t)rows * es, &p->ebe_out_r)) || (st = dalloc(p, 3 * (size_t)rows * es, &p->ebe_out_q)))
    return st;
  CK(cudaMemcpy(p->ebe_row_node, rnode.data(), rows * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_scale, scale.data(), rows * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_blocks, pk.blocks.data(), pk.blocks.size() * sizeof(EbeBlock), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_blob, pk.blob.data(), pk.blob.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_blk_nodes, pk.nodes.data(), pk.nodes.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->ebe_blk_rows, pk.rows.data(), pk.rows.size() * sizeof(int), cudaMemcpyHostToDevice));
  p->ebe_nblocks = (int)pk.blocks.size();
  p->ebe_smem = (pk.smem + 127) & ~127;  // one pipeline stage
  p->ebe_rows = (int)rows;
  return DDFD_OK;
}

}  // namespace

namespace ddfd {
namespace host {

int build_ebe(ddfd_problem *p) {
  const int a = p->a, b = p->b, n = p->n;
  const int fm = b - a - 1;  // rows per axis
  const long long rows = (long long)fm * fm * fm;
  const long long cubes = (long long)(b - a) * (b - a) * (b - a);
  const long long ntet = 6 * cubes;
  if (ntet > (1LL << 31) / 4) return fail(p, DDFD_E_ARG, "FEM mesh too large for the element path");
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  std::vector<int> tnode((size_t)ntet * 4);
  std::vector<double> tgrad((size_t)ntet * 12);
  std::vector<int> rptr((size_t)rows + 1, 0);
  std::vector<double> mass((size_t)rows, 0.0);
  auto off = [&](int i, int j, int k) { return (int)(i + (long long)p->px * (j + (long long)n * k)); };
  auto rowof = [&](int i, int j, int k) -> long long {
    if (i <= a || i >= b || j <= a || j >= b || k <= a || k >= b) return -1;
    return (i - a - 1) + (long long)fm * ((j - a - 1) + (long long)fm * (k - a - 1));
  };
  long long t = 0;
  for (int k = a; k < b; ++k)
    for (int j = a; j < b; ++j)
      for (int i = a; i < b; ++i)
        for (const auto &pm : perms) {
          int v[4][3] = {{i, j, k}};
          for (int q = 0; q < 3; ++q) {
            for (int d = 0; d < 3; ++d) v[q + 1][d] = v[q][d];
            v[q + 1][pm[q]] += 1;
          }
          double A[4][4], C[4][4];
          for (int q = 0; q < 4; ++q) {
            A[q][0] = 1.0;
            for (int d = 0; d < 3; ++d) A[q][d + 1] = v[q][d] * p->h;
          }
          if (!invert4(A, C)) return fail(p, DDFD_E_ARG, "degenerate tetrahedron in the FEM mesh");
          double e1[3], e2[3], e3[3];
          for (int d = 0; d < 3; ++d) {
            e1[d] = A[1][d + 1] - A[0][d + 1];
            e2[d] = A[2][d + 1] - A[0][d + 1];
            e3[d] = A[3][d + 1] - A[0][d + 1];
          }
          const double vol = std::fabs(e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                                       e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) / 6.0;
          const double sv = std::sqrt(vol);
          for (int q = 0; q < 4; ++q) {
            tnode[t * 4 + q] = off(v[q][0], v[q][1], v[q][2]);
            for (int d = 0; d < 3; ++d) tgrad[t * 12 + q * 3 + d] = sv * C[d + 1][q];
            const long long r = rowof(v[q][0], v[q][1], v[q][2]);
            if (r >= 0) {
              rptr[r + 1]++;
              mass[r] += vol / 4.0;
            }
          }
          ++t;
        }
  for (long long r = 0; r < rows; ++r) rptr[r + 1] += rptr[r];
  const long long ninc = rptr[rows];
  std::vector<int> itet((size_t)ninc), iloc((size_t)ninc), fillp(rptr.begin(), rptr.end() - 1), rnode((size_t)rows);
  std::vector<double> scale((size_t)rows);
  for (t = 0; t < ntet; ++t)
    for (int q = 0; q < 4; ++q) {
      const int o = tnode[t * 4 + q];
      const int i = (int)(o % p->px), j = (int)((o / p->px) % n), k = (int)(o / ((long long)p->px * n));
      const long long r = rowof(i, j, k);
      if (r >= 0) {
        itet[fillp[r]] = (int)t;
        iloc[fillp[r]++] = q;
      }
    }
  for (int k = a + 1; k < b; ++k)
    for (int j = a + 1; j < b; ++j)
      for (int i = a + 1; i < b; ++i) {
        const long long r = rowof(i, j, k);
        rnode[r] = off(i, j, k);
        scale[r] = p->h * p->h / mass[r];
      }
  std::vector<double> rpos((size_t)rows * 3);
  for (int k = a + 1; k < b; ++k)
    for (int j = a + 1; j < b; ++j)
      for (int i = a + 1; i < b; ++i) {
        const long long r = rowof(i, j, k);
        rpos[3 * r] = i;
        rpos[3 * r + 1] = j;
        rpos[3 * r + 2] = k;
      }
  return upload_ebe(p, rows, ntet, tnode, tgrad, rptr, itet, iloc, rnode, scale, rpos);
}

// Explicit refined FEM mesh (fem_kind = DDFD_FEM_MESH): node coordinates
// (new nodes as midpoints of their parents, in FP64), per-tet sqrt|K| g,
// the incidences of the FEM rows -- the grid nodes strictly inside the cube in
// the order of build_ebe, then the new nodes -- with their lumped masses, the
// masses of every free node, and the new nodes' field and coefficient arrays.
int build_mesh(ddfd_problem *p) {
  const int a = p->a, b = p->b, n = p->n;
  const long long n3 = (long long)n * n * n;
  const int fm = b - a - 1;
  const long long grid_rows = (long long)fm * fm * fm;
  const long long rows = grid_rows + p->n_new;
  const long long ntet = (long long)p->mesh_tets.size() / 4;
  if (p->cs + (long long)p->n_new >= (1LL << 31) || 4 * ntet >= (1LL << 31))
    return fail(p, DDFD_E_ARG, "refined mesh too large for 32-bit node offsets");
  std::vector<double> X((size_t)p->n_new * 3);
  auto xyz = [&](long long v, double out[3]) {
    if (v < n3) {
      out[0] = (double)(v % n) * p->h;
      out[1] = (double)((v / n) % n) * p->h;
      out[2] = (double)(v / ((long long)n * n)) * p->h;
    } else {
      for (int d = 0; d < 3; ++d) out[d] = X[(size_t)(v - n3) * 3 + d];
    }
  };
  const double lo = (p->f0 - 1e-9) * p->h, hi = (p->f0 + p->nf - 1 + 1e-9) * p->h;
  for (int e = 0; e < p->n_new; ++e) {
    double u[3], w[3];
    xyz(p->mesh_parents[2 * e], u);
    xyz(p->mesh_parents[2 * e + 1], w);
    for (int d = 0; d < 3; ++d) {
      X[(size_t)e * 3 + d] = 0.5 * (u[d] + w[d]);
      if (!(X[(size_t)e * 3 + d] >= lo && X[(size_t)e * 3 + d] <= hi))
        return fail(p, DDFD_E_ARG, "mesh: new node " + std::to_string(e) + " outside the free box");
    }
  }
  auto in_cube = [&](long long v) {
    const long long i = v % n, j = (v / n) % n, k = v / ((long long)n * n);
    return i >= a && i <= b && j >= a && j <= b && k >= a && k <= b;
  };
  auto rowof = [&](long long v) -> long long {
    if (v >= n3) return grid_rows + (v - n3);
    const long long i = v % n, j = (v / n) % n, k = v / ((long long)n * n);
    if (i <= a || i >= b || j <= a || j >= b || k <= a || k >= b) return -1;
    return (i - a - 1) + (long long)fm * ((j - a - 1) + (long long)fm * (k - a - 1));
  };
  auto off = [&](long long v) -> int {
    if (v >= n3) return (int)(p->cs + (v - n3));
    const long long i = v % n, j = (v / n) % n, k = v / ((long long)n * n);
    return (int)(i + (long long)p->px * (j + (long long)n * k));
  };
  std::vector<int> tnode((size_t)ntet * 4), rptr((size_t)rows + 1, 0);
  std::vector<double> tgrad((size_t)ntet * 12), mass((size_t)rows, 0.0);
  double vol_sum = 0.0;
  for (long long t = 0; t < ntet; ++t) {
    double A[4][4], C[4][4];
    for (int q = 0; q < 4; ++q) {
      const long long v = p->mesh_tets[t * 4 + q];
      if (v < n3 && !in_cube(v)) return fail(p, DDFD_E_ARG, "mesh: a grid node outside the FEM cube");
      double x[3];
      xyz(v, x);
      A[q][0] = 1.0;
      for (int d = 0; d < 3; ++d) A[q][d + 1] = x[d];
    }
    if (!invert4(A, C)) return fail(p, DDFD_E_ARG, "mesh: degenerate tetrahedron");
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = A[1][d + 1] - A[0][d + 1];
      e2[d] = A[2][d + 1] - A[0][d + 1];
      e3[d] = A[3][d + 1] - A[0][d + 1];
    }
    const double vol = std::fabs(e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                                 e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) / 6.0;
    vol_sum += vol;
    const double sv = std::sqrt(vol);
    for (int q = 0; q < 4; ++q) {
      const long long v = p->mesh_tets[t * 4 + q];
      tnode[t * 4 + q] = off(v);
      for (int d = 0; d < 3; ++d) tgrad[t * 12 + q * 3 + d] = sv * C[d + 1][q];
      const long long r = rowof(v);
      if (r >= 0) {
        rptr[r + 1]++;
        mass[r] += vol / 4.0;
      }
    }
  }
  const double cube = std::pow((b - a) * p->h, 3);
  if (std::fabs(vol_sum - cube) > 1e-9 * cube)
    return fail(p, DDFD_E_ARG, "mesh: the tetrahedra do not fill the FEM cube");
  for (long long r = 0; r < rows; ++r) {
    if (!(mass[r] > 0.0)) return fail(p, DDFD_E_ARG, "mesh: a FEM row without elements");
    rptr[r + 1] += rptr[r];
  }
  const long long ninc = rptr[rows];
  std::vector<int> itet((size_t)ninc), iloc((size_t)ninc), fillp(rptr.begin(), rptr.end() - 1), rnode((size_t)rows);
  std::vector<double> scale((size_t)rows);
  for (long long t = 0; t < ntet; ++t)
    for (int q = 0; q < 4; ++q) {
      const long long r = rowof(p->mesh_tets[t * 4 + q]);
      if (r >= 0) {
        itet[fillp[r]] = (int)t;
        iloc[fillp[r]++] = q;
      }
    }
  for (long long k = a + 1; k < b; ++k)
    for (long long j = a + 1; j < b; ++j)
      for (long long i = a + 1; i < b; ++i) {
        const long long v = i + n * (j + n * k);
        rnode[rowof(v)] = off(v);
      }
  for (int e = 0; e < p->n_new; ++e) rnode[grid_rows + e] = off(n3 + e);
  for (long long r = 0; r < rows; ++r) scale[r] = p->h * p->h / mass[r];
  // lumped masses of the free nodes: grid free nodes, then the new nodes
  std::vector<double> mfree((size_t)p->n_free);
  for (long long f = 0; f < p->n_free_grid; ++f) {
    const long long li = f % p->nf, lj = (f / p->nf) % p->nf, lk = f / ((long long)p->nf * p->nf);
    mfree[f] = mass[rowof((p->f0 + li) + n * ((p->f0 + lj) + (long long)n * (p->f0 + lk)))];
  }
  for (int e = 0; e < p->n_new; ++e) mfree[p->n_free_grid + e] = mass[grid_rows + e];
  std::vector<double> rpos((size_t)rows * 3);
  for (long long k = a + 1; k < b; ++k)
    for (long long j = a + 1; j < b; ++j)
      for (long long i = a + 1; i < b; ++i) {
        const long long r = rowof(i + n * (j + n * k));
        rpos[3 * r] = (double)i;
        rpos[3 * r + 1] = (double)j;
        rpos[3 * r + 2] = (double)k;
      }
  for (int e = 0; e < p->n_new; ++e)
    for (int d = 0; d < 3; ++d) rpos[3 * (grid_rows + e) + d] = X[(size_t)e * 3 + d] / p->h;
  // grid rows whose elements are the 24 untouched Kuhn tets take the block stencil
  std::vector<unsigned char> stencil;
  kuhn_stencil_rows(grid_rows, n, rptr.data(), itet.data(), p->mesh_tets.data(), &stencil);
  int st;
  if ((st = upload_ebe(p, rows, ntet, tnode, tgrad, rptr, itet, iloc, rnode, scale, rpos, &stencil))) return st;
  const size_t es = p->esz, xb = 3 * (size_t)std::max(p->n_new, 1) * es;
  if ((st = dalloc_t(p, (size_t)p->n_free, &p->mass_free)) || (st = dalloc(p, xb, &p->X[0])) ||
      (st = dalloc(p, xb, &p->X[1])) || (st = dalloc(p, xb, &p->xcoef)) ||
      (!p->fonly && ((st = dalloc(p, xb, &p->XMu[0])) || (st = dalloc(p, xb, &p->XMu[1])))))
    return st;
  CK(cudaMemcpy(p->mass_free, mfree.data(), p->n_free * sizeof(double), cudaMemcpyHostToDevice));
  for (int q = 0; q < 2; ++q) {
    CK(cudaMemset(p->X[q], 0, xb));
    if (p->XMu[q]) CK(cudaMemset(p->XMu[q], 0, xb));
  }
  CK(cudaMemset(p->xcoef, 0, xb));
  return DDFD_OK;
}

}  // namespace host
}  // namespace ddfd
