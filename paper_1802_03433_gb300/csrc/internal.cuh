// Internal declarations of libfea (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fea.h"
#include "devcommon.cuh"

namespace fea {

// A named NVTX range over a scope (pattern build, assembly, backward, batch
// launch): visible in a profiler's timeline; without one attached the calls
// return at once.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
fea_status fail(fea_status st, const std::string& msg);
fea_status cuda_fail(cudaError_t e, const char* what);

#define FEA_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e__ = (call);                                 \
    if (e__ != cudaSuccess) return ::fea::cuda_fail(e__, #call); \
  } while (0)

#define FEA_TRY(call)                   \
  do {                                  \
    fea_status s__ = (call);            \
    if (s__ != FEA_OK) return s__;      \
  } while (0)

// ------------------------------------------------------------------ handle
// Scalar-dof structures of one element order, shared by the scalar forms and
// (for P1) by elasticity.
struct Base {
  int nb = 0;               // local scalar dofs per element: 4 (P1) or 10 (P2)
  int64_t nsd = 0;          // number of scalar dofs
  int32_t* edof = nullptr;  // [nb][E] element -> scalar dof (P1: aliases mesh tets)
  bool own_edof = false;
  int32_t* rp = nullptr;    // [nsd + 1] scalar CSR row pointer
  int32_t* ci = nullptr;    // [nnz] scalar CSR columns
  int64_t nnz = 0;
  int32_t* inc_ptr = nullptr;  // [nsd + 1] dof -> incidences
  int32_t* inc = nullptr;      // [E * nb] incidence = e * nb + a, ascending e per dof
  uint8_t* slot = nullptr;     // [E * nb][SW] slot of each local column within the row
  int slot_width = 0;          // SW: 4 (P1) or 16 (P2)
  int max_row = 0;             // longest scalar row
  int32_t* ipos = nullptr;     // [nb][E] incidence index of (element e, local dof a)
  int32_t* emap = nullptr;     // [E][nb][nb] CSR position of local (a, b) (built on demand)
  int64_t nlong = 0;           // rows of more than 255 entries: their slot bytes are not used; the
  int32_t* long_rows = nullptr;  // local-row scatter adds them with k_long_rows (list, any order)
};

// Local rows are stored in incidence order: local row (e, a[, comp]) of the
// element with incidence index i = ipos[a][e] lives at row i * ndpn + comp of
// a buffer whose rows are lstride(nl, bytes) values apart (devcommon.cuh).

// Chunked scatter (chunks.cu, elast_chunk.cu, scalar_chunk.cu): the elements
// are grouped into spatially compact chunks (whole cells of a grid over the
// mesh's bounding box, visited in Morton order, at most CHUNK_MAX_ELEMS or
// CHUNK_MAX_ELEMS_P2 elements each).  One CTA assembles one chunk: the local
// entries of its elements are added as fixed-point integers into
// shared-memory accumulators, one block (3 x 3 for elasticity, one entry for
// scalar forms) per scalar dof pair ("slot") that the chunk's elements
// couple.  A slot whose every contributing element lies in
// the chunk is "owned" and written straight to the CSR values; the others are
// written as one FP64 partial sum per chunk and added, in chunk order, by a
// second kernel over the shared couplings.
constexpr int CHUNK_MAX_ELEMS = 384;     // P1 (scalar and vector)
constexpr int CHUNK_MAX_ELEMS_P2 = 128;  // P2: 55 dof pairs per element
// The elasticity chunk kernel stages a chunk's element ids and its ten rows of
// dof-pair slots in shared memory (rows of CHUNK_STAGE_E entries: the largest
// chunk plus the slack of rounding its bulk copies out to 16-byte boundaries),
// with the copies' mbarrier: CHUNK_STAGE_BYTES on top of its accumulators.
constexpr int CHUNK_STAGE_E = CHUNK_MAX_ELEMS + 8;
constexpr int CHUNK_STAGE_BYTES = CHUNK_STAGE_E * 4 + 10 * CHUNK_STAGE_E * 2 + 16;

// Index of the local dof pair (a, b), a <= b, of an element with nb local
// dofs: the nb diagonal pairs (the dof slots) first, then the pairs a < b in
// lexicographic order.
__host__ __device__ constexpr int pair_index(int nb, int a, int b) {
  return a == b ? a : nb + a * (nb - 1) - a * (a - 1) / 2 + (b - a - 1);
}

struct Chunks {
  int nb = 0, npair = 0, ndpn = 0;  // local scalar dofs, dof pairs per element, dofs per scalar dof
  int64_t nchunk = 0, nslot = 0, nnode_slot = 0;
  int max_slots = 0, max_nodes = 0;
  int hbits = 0;                 // ceil(log2(most elements contributing to one slot of a chunk))
  int32_t* cptr = nullptr;       // [nchunk + 1] element offsets into celem
  int32_t* celem = nullptr;      // [E] element ids, chunk by chunk
  uint16_t* eslot = nullptr;     // [npair][estride] (chunk order) slot of each local dof pair k =
                                 // pair_index(a, b) of the element (k < nb: the dof slot of local dof k);
                                 // bit 15 set when dof(a) > dof(b) (the slot holds the transposed block)
  int64_t estride = 0;           // row stride of eslot: E rounded up to 8, so every row starts 16-byte aligned
                                 // (celem and eslot have 16 bytes of padding past their ends, so bulk copies
                                 // rounded up to 16 bytes stay inside them)
  int32_t* sptr = nullptr;       // [nchunk + 1] slot offsets; each chunk's node slots come first
  int32_t* nptr = nullptr;       // [nchunk + 1] node-slot offsets
  int4* srec = nullptr;          // [nslot] {U, W, Li | Lj << 16, partial index or -1 when owned}: the
                                 // CSR position of entry (3i, 3j) and of (3j, 3i), the lengths of rows
                                 // 3i and 3j, for the slot's node pair i <= j
  int2* nrec = nullptr;          // [nnode_slot] {scalar dof, load partial index or -1 when owned}
  // couplings shared by several chunks: the partial sums of group g (one per
  // chunk that touches it) are partials gptr[g] .. gptr[g + 1] - 1, in chunk
  // order; a shared slot's record holds the index of its partial
  int64_t npart = 0, ngroup = 0;
  int32_t* gptr = nullptr;       // [ngroup + 1]
  int4* grec = nullptr;          // [ngroup] {U, W, Li | Lj << 16, 0}
  int64_t nnpart = 0, nngroup = 0;
  int32_t* ngptr = nullptr;      // [nngroup + 1]
  int32_t* ngnode = nullptr;     // [nngroup] node id
  int64_t niso = 0;
  int32_t* iso = nullptr;        // [niso] nodes of no element (their load entries are zero)
};

// The dof-level CSR pattern of (order, dofs per node).
struct Pattern {
  int order = 0, ndpn = 0;
  int64_t ndof = 0, nnz = 0;
  int32_t* row_ptr = nullptr;
  int32_t* col_idx = nullptr;
  bool own = false;           // ndpn == 1 aliases the Base arrays
  int rows_per_tile = 0;      // gather tile height (rows per CTA)
  int64_t max_tile_nnz = 0;   // largest CSR span of one tile
  // Overlap of element computation and scatter: the elements are processed
  // in `stages` consecutive chunks; the row tiles whose last element lies in
  // chunk k are listed in tile_list[stage_ptr[k] .. stage_ptr[k + 1]).
  int stages = 0;
  int64_t chunk = 0;
  int32_t* tile_list = nullptr;
  std::vector<int64_t> stage_ptr;
  // Tile classes of the sequential scatter: tiles whose CSR span is at most
  // `light_span` (the short rows) run in their own launch with a smaller
  // shared-memory allocation and a lighter kernel, so more CTAs fit per SM.
  int32_t* class_list = nullptr;   // heavy tiles, then light tiles
  int64_t n_heavy = 0, n_light = 0;
  int64_t heavy_span = 0, light_span = 0;
  // Tile-interleaved local rows (scalar patterns, gather_tiled.cuh): row tile
  // t owns positions tile_base[t] .. tile_base[t] + steps[t] * S_t, S_t = its
  // row count rounded up to 4; the k-th contribution (incidence) of its row
  // r0 + j sits at position tile_base[t] + k * S_t + j, so each step of a
  // tile is one contiguous block that one bulk copy moves.  Positions of rows
  // with fewer than steps[t] contributions stay unused (padding).
  int32_t* tpos = nullptr;        // [nb][E] position of local row (e, a)
  uint8_t* tslot = nullptr;       // [npos][SW] column slots at each position
  int64_t* tile_base = nullptr;   // [ntiles]
  int32_t* tile_steps = nullptr;  // [ntiles]
  int64_t npos = 0;               // positions, padding included (0: layout not built)
  Chunks* chunks = nullptr;       // chunked scatter (P1 vector pattern; built on first use)
  bool chunks_failed = false;     // the chunk structures cannot be built for this mesh
};

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};


}  // namespace fea

struct fea_mesh {
  const double* x = nullptr;
  const double* y = nullptr;
  const double* z = nullptr;
  int64_t n_nodes = 0;
  int64_t n_elems = 0;
  int nvert = 4;            // 4: tetrahedra, 3: triangles (z unused)
  int32_t* tets = nullptr;  // [nvert][E] owned copy
  int* err = nullptr;       // device error word
  fea::Base* base[3] = {nullptr, nullptr, nullptr};          // by order
  fea::Pattern* pat[3][4] = {{nullptr}};                     // by order, ndpn
  fea::Scratch lm, fl;      // local matrices / local loads of the last assembly
  fea::Scratch gxs;         // per-incidence vertex gradients of the last backward
  fea::Scratch part, npart; // chunked scatter: FP64 partial sums of shared couplings / of shared loads
  fea::Scratch bc;          // Dirichlet marks and values (fea_dirichlet)
  fea::Scratch cg;          // CG vectors, partial sums and state (fea_cg)
  cudaStream_t solve_stream = nullptr;  // stream the CG iteration graph is captured on
  cudaEvent_t solve_ev = nullptr;
  int stages = 1;           // element chunks overlapped with the scatter (1 = no overlap)
  int tile_classes = -1;    // sequential scatter: 0 one deep launch, 1 heavy/light split, 2 one light
                            // launch, -1 automatic (2 when the pattern mixes long and short rows, else 0)
  cudaStream_t side = nullptr;             // scatter stream of the overlapped path
  cudaEvent_t chunk_ev[17] = {nullptr};    // chunk done (<= 16 stages) + join
  int tiled_stages = 0;     // bulk-copy scatter stages per CTA (2..4), 0 automatic
  int scatter = 0;          // FEA_SCATTER_*: 0 automatic, 1 local rows through HBM, 2 chunked fixed point
  int load_split = -1;      // scalar forms: 0 fused element kernel; 1 matrix kernel then load kernel;
                            // 2 load kernel on the side stream, concurrent with the matrix kernel;
                            // 3 one kernel with matrix warps and load warps; -1 automatic (3 for
                            // FP64 P2 with the sine load, else 0)
  bool profile = false;     // record phase events in fea_assemble
  bool profiled = false;    // events of a call are pending
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};

namespace fea {

// pattern.cu
fea_status build_base(fea_mesh* m, int order, cudaStream_t s);
fea_status build_pattern(fea_mesh* m, int order, int ndpn, cudaStream_t s);
fea_status build_emap(fea_mesh* m, int order, cudaStream_t s);
fea_status build_stages(fea_mesh* m, Pattern* P, int stages, cudaStream_t s);
fea_status validate_connectivity(fea_mesh* m, cudaStream_t s);
void free_base(Base* b);
void free_pattern(Pattern* p);

// chunks.cu
fea_status build_chunks(fea_mesh* m, Pattern* P, cudaStream_t s);
void free_chunks(Chunks* c);

// elast_chunk.cu, scalar_chunk.cu
fea_status assemble_chunked(fea_mesh* m, Pattern* P, const fea_coeffs* co, const fea_quadrature* q, int load,
                            double* values, double* rhs, cudaStream_t s);
fea_status assemble_chunked_scalar(fea_mesh* m, Pattern* P, const fea_form* form, const fea_coeffs* co,
                                   const fea_quadrature* q, int load, double* values, double* rhs, cudaStream_t s);

// assemble.cu
fea_status assemble(fea_mesh* m, const fea_form* form, const fea_coeffs* co,
                    const fea_quadrature* q, double* values, double* rhs, cudaStream_t s);

// adjoint.cu
fea_status assemble_backward(fea_mesh* m, const fea_form* form, const fea_coeffs* co,
                             const fea_quadrature* q, const double* gv, const double* gf,
                             double* gk, double* gx, cudaStream_t s);

// argument checks shared by the assembly entry points (fea_api.cu): NULL
// pointers, order / kind / rule / precision / load codes, 8-byte alignment
// of the coefficient arrays
bool aligned(const void* p, size_t a);
fea_status check_form(const fea_mesh* m, const fea_form* f, const fea_coeffs* c, const fea_quadrature* q);

// Entry points other than fea_assemble read the one-byte column slots, which
// rows of more than 255 entries do not have: they refuse such meshes.
inline fea_status refuse_long_rows(const Base* B, const char* what) {
  if (B && B->nlong > 0)
    return fail(FEA_ERR_OVERFLOW, std::string(what) + ": rows of more than 255 entries are assembled by fea_assemble "
                                                      "only");
  return FEA_OK;
}

// scratch management (fea_api.cu)
fea_status ensure_scratch(Scratch& sc, size_t bytes);
fea_status read_and_clear_err(fea_mesh* m, cudaStream_t s);

}  // namespace fea
