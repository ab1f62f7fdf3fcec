// Host-side construction of the Kuhn P1 block stencil used by the step
// kernels.  The 24 Kuhn tetrahedra around an interior node (six per grid
// cube, 0 -> e_p0 -> e_p0+e_p1 -> (1,1,1) for each axis permutation p) are
// assembled at h = 1:
//   (D^T D)_{0,o} = sum_K |K| g_0 g_o^T    (P1 div-div, the Gauss-law term)
//   L_{0,o}       = sum_K |K| g_0 . g_o    (P1 Laplacian)
//   m_0           = sum_K |K| / 4          (lumped mass)
// and checked against what the FD region uses at the same node: the FE rows
// must be the 7-point Laplacian with m = h^3, so that FD and FE rows agree
// wherever the two regions overlap.  The div-div blocks must satisfy
// B_{-o} = B_o = B_o^T.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "ddfd_internal.h"

namespace ddfd {

bool invert4(const double A[4][4], double X[4][4]) {
  double M[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) M[r][c] = c < 4 ? A[r][c] : (c - 4 == r ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (std::fabs(M[piv][c]) < 1e-14) return false;
    if (piv != c)
      for (int q = 0; q < 8; ++q) std::swap(M[c][q], M[piv][q]);
    const double d = M[c][c];
    for (int q = 0; q < 8; ++q) M[c][q] /= d;
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        const double f = M[r][c];
        for (int q = 0; q < 8; ++q) M[r][q] -= f * M[c][q];
      }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) X[r][c] = M[r][c + 4];
  return true;
}

bool build_kuhn_blocks(KuhnBlocks *out, std::string *msg) {
  double B[27][9];
  double L[27];
  std::memset(B, 0, sizeof(B));
  std::memset(L, 0, sizeof(L));
  double mass = 0.0;
  auto oi = [](int dx, int dy, int dz) { return (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1)); };
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int cz = -1; cz <= 0; ++cz)
    for (int cy = -1; cy <= 0; ++cy)
      for (int cx = -1; cx <= 0; ++cx)
        for (const auto &p : perms) {
          int v[4][3] = {{cx, cy, cz}};
          for (int m = 0; m < 3; ++m) {
            for (int d = 0; d < 3; ++d) v[m + 1][d] = v[m][d];
            v[m + 1][p[m]] += 1;
          }
          int a = -1;
          for (int q = 0; q < 4; ++q)
            if (v[q][0] == 0 && v[q][1] == 0 && v[q][2] == 0) a = q;
          if (a < 0) continue;
          double A[4][4], C[4][4];
          for (int q = 0; q < 4; ++q) {
            A[q][0] = 1.0;
            for (int d = 0; d < 3; ++d) A[q][d + 1] = v[q][d];
          }
          if (!invert4(A, C)) {
            *msg = "singular Kuhn tetrahedron";
            return false;
          }
          double g[4][3];
          for (int q = 0; q < 4; ++q)
            for (int d = 0; d < 3; ++d) g[q][d] = C[d + 1][q];
          const double vol = 1.0 / 6.0;
          mass += vol / 4.0;
          for (int q = 0; q < 4; ++q) {
            const int o = oi(v[q][0], v[q][1], v[q][2]);
            for (int c = 0; c < 3; ++c)
              for (int d = 0; d < 3; ++d) B[o][c * 3 + d] += vol * g[a][c] * g[q][d];
            L[o] += vol * (g[a][0] * g[q][0] + g[a][1] * g[q][1] + g[a][2] * g[q][2]);
          }
        }
  const int pos[8][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
                         {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
  const double tol = 1e-12;
  if (std::fabs(mass - 1.0) > tol) {
    *msg = "Kuhn lumped mass of an interior node is not h^3";
    return false;
  }
  // FE Laplacian row must be the 7-point FD row: 6 at the centre, -1 on the axes.
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        const double want = nz == 0 ? 6.0 : (nz == 1 ? -1.0 : 0.0);
        if (std::fabs(L[oi(dx, dy, dz)] - want) > tol) {
          *msg = "Kuhn P1 Laplacian row differs from the 7-point FD row";
          return false;
        }
      }
  for (int q = 0; q < 8; ++q) {
    const int o = oi(pos[q][0], pos[q][1], pos[q][2]);
    const int mo = oi(-pos[q][0], -pos[q][1], -pos[q][2]);
    for (int e = 0; e < 9; ++e) {
      const int c = e / 3, d = e % 3;
      if (std::fabs(B[o][e] - B[mo][e]) > tol || std::fabs(B[o][e] - B[o][d * 3 + c]) > tol) {
        *msg = "Kuhn div-div blocks are not even and symmetric";
        return false;
      }
      out->B[q][e] = B[o][e];
    }
    out->lap[q] = L[o];
  }
  // only the 15 offsets 0, +-o of the table may carry a block
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        bool listed = false;
        for (int q = 0; q < 8; ++q)
          if ((dx == pos[q][0] && dy == pos[q][1] && dz == pos[q][2]) ||
              (dx == -pos[q][0] && dy == -pos[q][1] && dz == -pos[q][2]))
            listed = true;
        if (listed) continue;
        for (int e = 0; e < 9; ++e)
          if (std::fabs(B[oi(dx, dy, dz)][e]) > tol) {
            *msg = "Kuhn div-div couples an offset outside the 15-point table";
            return false;
          }
      }
  out->mass = mass;
  return true;
}

}  // namespace ddfd
