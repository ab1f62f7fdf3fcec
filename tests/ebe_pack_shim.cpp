// Host-only entry to the element-by-element block packer, for the CPU tests
// of its layout (compiled by tests/test_ebe_pack.py with the host compiler).
#include <cstring>

#include "ddfd_internal.h"

static ddfd::EbePack g_pack;

extern "C" int ebe_pack_run(long long n_rows, long long ntet, const int *tnode, const double *tgrad,
                            const int *rptr, const int *itet, const int *iloc, const double *rpos, int esz,
                            long long *sizes, char *err, int err_len, const unsigned char *use) {
  std::string m;
  if (!ddfd::pack_ebe_blocks(n_rows, ntet, tnode, tgrad, rptr, itet, iloc, rpos, esz, &g_pack, &m, use)) {
    std::strncpy(err, m.c_str(), err_len - 1);
    err[err_len - 1] = 0;
    return 1;
  }
  sizes[0] = (long long)g_pack.blocks.size();
  sizes[1] = (long long)g_pack.blob.size();
  sizes[2] = (long long)g_pack.nodes.size();
  sizes[3] = (long long)g_pack.rows.size();
  sizes[4] = g_pack.smem;
  return 0;
}

// blocks: [n_blocks][8] = blob, bytes, nt, nn, maxinc, nrows, node0, row0
extern "C" void ebe_pack_fetch(long long *blocks, unsigned char *blob, int *nodes, int *rows) {
  for (size_t i = 0; i < g_pack.blocks.size(); ++i) {
    const ddfd::EbeBlock &B = g_pack.blocks[i];
    const long long v[8] = {B.blob, B.bytes, B.nt, B.nn, B.maxinc, B.nrows, B.node0, B.row0};
    std::memcpy(blocks + 8 * i, v, sizeof(v));
  }
  std::memcpy(blob, g_pack.blob.data(), g_pack.blob.size());
  std::memcpy(nodes, g_pack.nodes.data(), g_pack.nodes.size() * sizeof(int));
  std::memcpy(rows, g_pack.rows.data(), g_pack.rows.size() * sizeof(int));
}

extern "C" long long ebe_pack_smem(long long nt, long long nn, long long maxinc, int esz) {
  return ddfd::ebe_block_smem(nt, nn, maxinc, esz);
}

// rows per block, shared-memory budget, padding code
extern "C" void ebe_pack_consts(int *v) {
  v[0] = ddfd::EBE_RB;
  v[1] = ddfd::EBE_SMEM_BUDGET;
  v[2] = ddfd::EBE_PAD;
}

// grid rows that are Kuhn block-stencil rows (1) or gathered (0)
extern "C" void ebe_kuhn_rows(long long n_grid_rows, int n, const int *rptr, const int *itet, const int *tet_ids,
                              unsigned char *out) {
  std::vector<unsigned char> v;
  ddfd::kuhn_stencil_rows(n_grid_rows, n, rptr, itet, tet_ids, &v);
  std::memcpy(out, v.data(), v.size());
}

// (D^T D)_{i,i+o} / h of the uniform Kuhn split, as the library assembles it
extern "C" int ebe_kuhn_blocks(double *B) {
  ddfd::KuhnBlocks kb;
  std::string m;
  if (!ddfd::build_kuhn_blocks(&kb, &m)) return 1;
  std::memcpy(B, kb.B, sizeof(kb.B));
  return 0;
}
