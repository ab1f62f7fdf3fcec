// Host packer of the staged element-by-element gather (see EbeBlock in
// ddfd_internal.h): orders the FEM rows by brick, cuts them into blocks that
// fit the shared-memory budget, and lays out each block's tets and incidences
// in the order the kernel reads them.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "ddfd_internal.h"

namespace ddfd {

namespace {

long long align16(long long b) { return (b + 15) & ~15LL; }

// Blob bytes of a block: gradients, local node ids, incidences.
long long blob_bytes(long long nt, long long maxinc, int esz) {
  return align16(nt * (12LL * esz + 8) + maxinc * EBE_RB * 2LL);
}

}  // namespace

long long ebe_block_smem(long long nt, long long nn, long long maxinc, int esz) {
  nt += nt & 1;
  // blob, node values [nn][4] (field components and s), per-tet divergence
  return blob_bytes(nt, maxinc, esz) + align16(nn * 4LL * esz) + align16(nt * (long long)esz);
}

void kuhn_stencil_rows(long long n_grid_rows, int n, const int *rptr, const int *itet, const int *tet_ids,
                       std::vector<unsigned char> *is_stencil) {
  const long long n3 = (long long)n * n * n;
  is_stencil->assign((size_t)n_grid_rows, 0);
  auto kuhn_tet = [&](long long t) {
    long long v[4][3];
    for (int q = 0; q < 4; ++q) {
      const long long id = tet_ids[4 * t + q];
      if (id < 0 || id >= n3) return false;  // a new node
      v[q][0] = id % n;
      v[q][1] = (id / n) % n;
      v[q][2] = id / ((long long)n * n);
    }
    // order the vertices by coordinate sum; a Kuhn path climbs one axis per step
    int ord[4] = {0, 1, 2, 3};
    std::sort(ord, ord + 4, [&](int x, int y) { return v[x][0] + v[x][1] + v[x][2] < v[y][0] + v[y][1] + v[y][2]; });
    int used = 0;
    for (int q = 0; q < 3; ++q) {
      int axis = -1, steps = 0;
      for (int d = 0; d < 3; ++d) {
        const long long dd = v[ord[q + 1]][d] - v[ord[q]][d];
        if (dd == 1) axis = d, ++steps;
        else if (dd != 0) return false;
      }
      if (steps != 1 || (used >> axis) & 1) return false;
      used |= 1 << axis;
    }
    return true;
  };
  for (long long r = 0; r < n_grid_rows; ++r) {
    if (rptr[r + 1] - rptr[r] != 24) continue;
    bool ok = true;
    for (int e = rptr[r]; e < rptr[r + 1] && ok; ++e) ok = kuhn_tet(itet[e]);
    (*is_stencil)[r] = ok ? 1 : 0;
  }
}

bool pack_ebe_blocks(long long n_rows, long long ntet, const int *tnode, const double *tgrad, const int *rptr,
                     const int *itet, const int *iloc, const double *rpos, int esz, EbePack *out, std::string *err,
                     const unsigned char *use) {
  out->blocks.clear();
  out->blob.clear();
  out->nodes.clear();
  out->rows.clear();
  out->smem = 0;
  // compact node ids: the distinct offsets in ascending order
  std::vector<int> uniq(tnode, tnode + 4 * ntet);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  std::vector<int> tnc((size_t)(4 * ntet));
  for (long long i = 0; i < 4 * ntet; ++i)
    tnc[i] = (int)(std::lower_bound(uniq.begin(), uniq.end(), tnode[i]) - uniq.begin());
  // rows in brick order (8 x 4 x 4 spacings, x fastest), then z, y, x inside
  std::vector<long long> order;
  order.reserve((size_t)n_rows);
  for (long long r = 0; r < n_rows; ++r)
    if (!use || use[r]) order.push_back(r);
  auto key = [&](long long r) {
    const double *x = rpos + 3 * r;
    return std::make_tuple(std::floor(x[2] / 4.0), std::floor(x[1] / 4.0), std::floor(x[0] / 8.0), x[2], x[1], x[0]);
  };
  std::stable_sort(order.begin(), order.end(), [&](long long u, long long v) { return key(u) < key(v); });

  std::vector<int> stampT((size_t)ntet, -1), candT((size_t)ntet, -1), locT((size_t)ntet, 0);
  std::vector<int> stampN(uniq.size(), -1), candN(uniq.size(), -1), locN(uniq.size(), 0);
  std::vector<int> bt, bn;           // the open block's tets and compact nodes
  std::vector<long long> br;         // and rows
  int bid = 0, serial = 0, maxinc = 0;
  std::vector<int> newT, newN;

  auto close_block = [&]() {
    std::sort(bt.begin(), bt.end());
    std::sort(bn.begin(), bn.end());
    for (size_t i = 0; i < bt.size(); ++i) locT[bt[i]] = (int)i;
    for (size_t i = 0; i < bn.size(); ++i) locN[bn[i]] = (int)i;
    const long long nt = (long long)bt.size() + (bt.size() & 1);
    EbeBlock B;
    B.blob = (long long)out->blob.size();
    B.bytes = (int)blob_bytes(nt, maxinc, esz);
    B.nt = (int)nt;
    B.nn = (int)bn.size();
    B.maxinc = maxinc;
    B.nrows = (int)br.size();
    B.node0 = (int)out->nodes.size();
    B.row0 = (int)out->rows.size();
    out->blob.resize(out->blob.size() + B.bytes, 0);
    unsigned char *base = out->blob.data() + B.blob;
    unsigned char *gp = base;
    uint16_t *np = reinterpret_cast<uint16_t *>(base + nt * 12LL * esz);
    uint16_t *ip = reinterpret_cast<uint16_t *>(base + nt * (12LL * esz + 8));
    for (size_t i = 0; i < bt.size(); ++i) {
      const long long t = bt[i];
      for (int q = 0; q < 12; ++q) {
        if (esz == 4) {
          const float v = (float)tgrad[12 * t + q];
          std::memcpy(gp + (i * 12 + q) * 4, &v, 4);
        } else {
          std::memcpy(gp + (i * 12 + q) * 8, &tgrad[12 * t + q], 8);
        }
      }
      for (int q = 0; q < 4; ++q) np[4 * i + q] = (uint16_t)locN[tnc[4 * t + q]];
    }
    // the padding tet (zero gradients) points at node 0
    std::fill(ip, ip + (size_t)maxinc * EBE_RB, EBE_PAD);
    for (size_t lr = 0; lr < br.size(); ++lr) {
      const long long r = br[lr];
      for (int e = rptr[r]; e < rptr[r + 1]; ++e)
        ip[(size_t)(e - rptr[r]) * EBE_RB + lr] = (uint16_t)((locT[itet[e]] << 2) | iloc[e]);
    }
    for (int c : bn) out->nodes.push_back(uniq[c]);
    for (long long r : br) out->rows.push_back((int)r);
    out->smem = std::max(out->smem, (int)ebe_block_smem(nt, B.nn, maxinc, esz));
    out->blocks.push_back(B);
    bt.clear();
    bn.clear();
    br.clear();
    maxinc = 0;
    ++bid;
  };

  for (long long r : order) {
    const int deg = rptr[r + 1] - rptr[r];
    for (int attempt = 0; attempt < 2; ++attempt) {
      ++serial;
      newT.clear();
      newN.clear();
      for (int e = rptr[r]; e < rptr[r + 1]; ++e) {
        const int t = itet[e];
        if (stampT[t] == bid || candT[t] == serial) continue;
        candT[t] = serial;
        newT.push_back(t);
        for (int q = 0; q < 4; ++q) {
          const int c = tnc[4 * (long long)t + q];
          if (stampN[c] == bid || candN[c] == serial) continue;
          candN[c] = serial;
          newN.push_back(c);
        }
      }
      const long long nt = (long long)(bt.size() + newT.size());
      const long long bytes = ebe_block_smem(nt, (long long)(bn.size() + newN.size()), std::max(maxinc, deg), esz);
      const bool fits = (long long)br.size() < EBE_RB && bytes <= EBE_SMEM_BUDGET && nt < (1 << 14);
      if (fits) break;
      if (br.empty()) {
        *err = "FEM row " + std::to_string(r) + " has too many elements for the gather's shared memory";
        return false;
      }
      close_block();  // and count again against the empty block
    }
    for (int t : newT) {
      stampT[t] = bid;
      bt.push_back(t);
    }
    for (int c : newN) {
      stampN[c] = bid;
      bn.push_back(c);
    }
    br.push_back(r);
    maxinc = std::max(maxinc, deg);
  }
  if (!br.empty()) close_block();
  return true;
}

}  // namespace ddfd
