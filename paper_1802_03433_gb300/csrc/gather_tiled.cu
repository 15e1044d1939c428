// Launchers of the bulk-copy scatter (gather_tiled.cuh).
#include <cuda_runtime.h>

#include <algorithm>

#include "gather_tiled.cuh"

namespace fea {
namespace {

template <int NB, typename LT, int STAGES>
fea_status tiled_one(const TiledArgs& G, cudaStream_t s, const int32_t* tiles, int64_t ntiles) {
  const size_t smem = Tiled<NB, LT>::smem_bytes(G.rows, G.span_cap, STAGES);
  if (smem > 227 * 1024) return fail(FEA_ERR_OVERFLOW, "row tile too large for the bulk-copy scatter");
  static size_t configured = 0;  // opt-in above the 48 KB default, once per instance
  if (smem > 48 * 1024 && smem > configured) {
    FEA_CUDA(cudaFuncSetAttribute(k_gather_tiled<NB, LT, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    configured = smem;
  }
  if (ntiles > 0) k_gather_tiled<NB, LT, STAGES><<<(unsigned)ntiles, G.rows, smem, s>>>(G, tiles);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

template <int NB, typename LT>
fea_status tiled_stages(const TiledArgs& G, cudaStream_t s, const int32_t* tiles, int64_t ntiles, int stages) {
  if (stages == 2) return tiled_one<NB, LT, 2>(G, s, tiles, ntiles);
  if (stages == 4) return tiled_one<NB, LT, 4>(G, s, tiles, ntiles);
  return tiled_one<NB, LT, 3>(G, s, tiles, ntiles);
}

template <int NB, typename LT>
size_t tiled_smem(int rows, int64_t span_cap, int stages) {
  return Tiled<NB, LT>::smem_bytes(rows, span_cap, stages);
}

}  // namespace

int tiled_stages_auto(int nb, bool mixed, int rows, int64_t span_cap) {
  static int per_sm = 0, reserved = 0;
  if (!per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 228 * 1024;
      reserved = 1024;
    }
  }
  int best = TILED_STAGES, best_ctas = 0;
  for (int st = 2; st <= TILED_MAX_STAGES; ++st) {
    const size_t smem = nb == 3    ? tiled_smem<3, double>(rows, span_cap, st)
                        : nb == 4  ? (mixed ? tiled_smem<4, float>(rows, span_cap, st)
                                            : tiled_smem<4, double>(rows, span_cap, st))
                                   : (mixed ? tiled_smem<10, float>(rows, span_cap, st)
                                            : tiled_smem<10, double>(rows, span_cap, st));
    if (smem > 227 * 1024) break;
    const int ctas = std::min<int>(per_sm / (int)(smem + reserved), 2048 / std::max(rows, 32));
    if (ctas > best_ctas) {  // ties keep the fewer stages
      best = st;
      best_ctas = ctas;
    }
  }
  return best;
}

fea_status launch_gather_tiled(int nb, bool mixed, const TiledArgs& G, cudaStream_t s, const int32_t* tiles,
                               int64_t ntiles, int stages) {
  if (stages <= 0) stages = tiled_stages_auto(nb, mixed, G.rows, G.span_cap);
  if (nb == 3 && !mixed) return tiled_stages<3, double>(G, s, tiles, ntiles, stages);
  if (nb == 4)
    return mixed ? tiled_stages<4, float>(G, s, tiles, ntiles, stages)
                 : tiled_stages<4, double>(G, s, tiles, ntiles, stages);
  if (nb == 10)
    return mixed ? tiled_stages<10, float>(G, s, tiles, ntiles, stages)
                 : tiled_stages<10, double>(G, s, tiles, ntiles, stages);
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
    FEA_TRY(launch_gather_tiled(B->nb, mixed, G, s, P->class_list, P->n_heavy, m->tiled_stages));
    G.span_cap = P->light_span;
    return launch_gather_tiled(B->nb, mixed, G, s, P->class_list + P->n_heavy, P->n_light, m->tiled_stages);
  }
  G.span_cap = P->max_tile_nnz;
  return launch_gather_tiled(B->nb, mixed, G, s, nullptr, (P->ndof + G.rows - 1) / G.rows, m->tiled_stages);
}

fea_status scatter_tiled_list(const fea_mesh* m, const Pattern* P, const Base* B, bool mixed, const void* Lm,
                              const void* Fl, double* values, double* rhs, const int32_t* tiles, int64_t ntiles,
                              cudaStream_t s) {
  if (!P->tpos || !P->tslot || !P->tile_base || !P->tile_steps || P->npos <= 0)
    return fail(FEA_ERR_STATE, "bulk-copy scatter without a tiled layout");
  TiledArgs G = tiled_args(m, P, B, Lm, Fl, values, rhs);
  G.span_cap = P->max_tile_nnz;
  return launch_gather_tiled(B->nb, mixed, G, s, tiles, ntiles, m->tiled_stages);
}

}  // namespace fea
