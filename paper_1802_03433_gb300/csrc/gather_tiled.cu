// Launchers of the bulk-copy scatter (gather_tiled.cuh).
#include <cuda_runtime.h>

#include "gather_tiled.cuh"

namespace fea {
namespace {

template <int NB, typename LT>
fea_status tiled_one(const TiledArgs& G, cudaStream_t s, const int32_t* tiles, int64_t ntiles) {
  const size_t smem = Tiled<NB, LT>::smem_bytes(G.rows, G.span_cap);
  if (smem > 227 * 1024) return fail(FEA_ERR_OVERFLOW, "row tile too large for the bulk-copy scatter");
  static size_t configured = 0;  // opt-in above the 48 KB default, once per instance
  if (smem > 48 * 1024 && smem > configured) {
    FEA_CUDA(cudaFuncSetAttribute(k_gather_tiled<NB, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = smem;
  }
  if (ntiles > 0) k_gather_tiled<NB, LT><<<(unsigned)ntiles, G.rows, smem, s>>>(G, tiles);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

}  // namespace

fea_status launch_gather_tiled(int nb, bool mixed, const TiledArgs& G, cudaStream_t s, const int32_t* tiles,
                               int64_t ntiles) {
  if (nb == 3 && !mixed) return tiled_one<3, double>(G, s, tiles, ntiles);
  if (nb == 4) return mixed ? tiled_one<4, float>(G, s, tiles, ntiles) : tiled_one<4, double>(G, s, tiles, ntiles);
  if (nb == 10) return mixed ? tiled_one<10, float>(G, s, tiles, ntiles) : tiled_one<10, double>(G, s, tiles, ntiles);
  return fail(FEA_ERR_ARG, "no bulk-copy scatter for this element");
}

bool use_tiled(const fea_mesh* m, const Pattern* P) {
  return P && P->npos > 0 && P->ndpn == 1 && (m->tile_classes == -1 || m->tile_classes == 3);
}

namespace {
TiledArgs tiled_args(const fea_mesh* m, const Pattern* P, const Base* B, const void* Lm, const void* Fl,
                     double* values, double* rhs) {
  TiledArgs G{};
  G.ndof = P->ndof;
  G.rows = P->rows_per_tile;
  G.row_ptr = P->row_ptr;
  G.inc_ptr = B->inc_ptr;
  G.tile_base = P->tile_base;
  G.tile_steps = P->tile_steps;
  G.tslot = P->tslot;
  G.Lm = Lm;
  G.Fl = Fl;
  G.values = values;
  G.rhs = rhs;
  G.err = m->err;
  return G;
}
}  // namespace

fea_status scatter_tiled(const fea_mesh* m, const Pattern* P, const Base* B, bool mixed, const void* Lm,
                         const void* Fl, double* values, double* rhs, cudaStream_t s) {
  if (!P->tpos || !P->tslot || !P->tile_base || !P->tile_steps || P->npos <= 0)
    return fail(FEA_ERR_STATE, "bulk-copy scatter without a tiled layout");
  TiledArgs G = tiled_args(m, P, B, Lm, Fl, values, rhs);
  if (P->class_list && P->n_heavy > 0 && P->n_light > 0) {
    // long-row tiles, then short-row tiles with a smaller accumulator (more CTAs per SM)
    G.span_cap = P->heavy_span;
    FEA_TRY(launch_gather_tiled(B->nb, mixed, G, s, P->class_list, P->n_heavy));
    G.span_cap = P->light_span;
    return launch_gather_tiled(B->nb, mixed, G, s, P->class_list + P->n_heavy, P->n_light);
  }
  G.span_cap = P->max_tile_nnz;
  return launch_gather_tiled(B->nb, mixed, G, s, nullptr, (P->ndof + G.rows - 1) / G.rows);
}

fea_status scatter_tiled_list(const fea_mesh* m, const Pattern* P, const Base* B, bool mixed, const void* Lm,
                              const void* Fl, double* values, double* rhs, const int32_t* tiles, int64_t ntiles,
                              cudaStream_t s) {
  if (!P->tpos || !P->tslot || !P->tile_base || !P->tile_steps || P->npos <= 0)
    return fail(FEA_ERR_STATE, "bulk-copy scatter without a tiled layout");
  TiledArgs G = tiled_args(m, P, B, Lm, Fl, values, rhs);
  G.span_cap = P->max_tile_nnz;
  return launch_gather_tiled(B->nb, mixed, G, s, tiles, ntiles);
}

}  // namespace fea
