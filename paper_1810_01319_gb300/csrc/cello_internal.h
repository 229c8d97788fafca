// Internal types shared by the host orchestration and the kernel translation
// units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cello.h"

namespace cello {

constexpr int kGhosts = 4;
constexpr int kFields = 5;
constexpr int kAdjPencils = 4;       // pencils per adjoint-sweep CTA

// Launch variants of the PPM sweep: pencils per CTA, the minimum number of
// resident CTAs per SM the register allocation is bounded for, and the
// schedule (static: one CTA per item; persistent: one resident wave of CTAs
// pulling items from a device counter).  The autotuner times them.
struct SweepVariant {
  int pencils;       // pencils per CTA (the CTA size of the streaming form)
  int min_blocks;    // resident CTAs per SM the register bound is set for
  bool persistent;   // work-counter schedule over a resident grid
  bool stream;       // register-streaming form (sweep_stream_kernel)
  int vec;           // streaming form moving x pencils four cells at a time, staged by cp.async (3), or not (0)
};
int sweep_variant_count_f32();
int sweep_variant_count_f64();
SweepVariant sweep_variant_f32(int v);
SweepVariant sweep_variant_f64(int v);

// Neighbour kinds of the 27-entry table.
enum NbKind : int8_t { kSame = 0, kCoarse = 1, kFine = 2, kBoundary = 3 };

// Read-only view of the device-resident block table.
struct DevMesh {
  int n, g, N;            // cells per block edge, ghosts, padded edge
  int max_level;
  int root[3];
  int bc[3];              // 0 periodic, 1 outflow
  double dx0;             // cell width at level 0
  double gamma;
  int riemann;            // CELLO_RIEMANN_TWO_SHOCK or CELLO_RIEMANN_HLLC
  int steepen;            // contact steepening of the density edge values
  int nf;                 // fields per cell: 5, or 6 with the dual-energy formalism's rho e
  int B;                  // leaves
  const int4* leaf;       // (level, i, j, k)
  const int8_t* kind;     // [B][27]
  const int* idx;         // [B][27]
  const int* fine8;       // [B][27][8]
  const int* face_slot;   // [B][6] flux-register slot of each face or -1
  unsigned* err;          // error word: bit 0 set by the reduction on a non-finite or non-positive state
};

// Face order used by registers and corrections: -x, +x, -y, +y, -z, +z.
__host__ __device__ inline int face_dir(int axis, int side) {
  int d[3] = {0, 0, 0};
  d[axis] = side;
  return (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1);
}

// One coarse face that touches four finer leaves.
struct CoarseFace {
  int leaf;       // coarse leaf
  int axis, side; // face
  int cslot;      // register slot of the coarse flux
  int fslot[4];   // register slots of the fine fluxes, index o2*2 + o1
};

// Unsigned division by a launch-time constant as a multiply-high and shift
// (Granlund & Montgomery): valid for dividends below 2^31.
struct FastDiv {
  unsigned d, m, s;
  __host__ __device__ static FastDiv make(unsigned d) {
    FastDiv f;
    f.d = d;
    f.s = 0;
    while ((1u << f.s) < d) ++f.s;
    f.m = (unsigned)((((unsigned long long)1 << 32) * ((1ull << f.s) - d)) / d + 1);
    return f;
  }
  __device__ __forceinline__ unsigned div(unsigned x) const { return (__umulhi(x, m) + x) >> s; }
};

struct SweepParams {
  void* U;
  int leaf0, nleaf;        // leaves [leaf0, leaf0 + nleaf)
  int axis;
  int a0, a1, b0, b1;      // transverse ranges (padded coordinates)
  int tiles_per_leaf;      // set by the launcher from the variant's pencils per CTA
  const double* dt;        // device scalar
  double* reg;             // flux registers (may be null)
  unsigned* work;          // work counter for persistent variants (device, 4 bytes)
  int n_items;             // set by the launcher
  int variant;             // index into the sweep variants of the precision
  FastDiv div_tiles, div_cb;   // set by the launcher: by tiles_per_leaf and by the B-range length
};

struct AdjSweepParams {
  const void* U;           // state entering the forward sweep (ghosts refreshed)
  void* lam;               // adjoint, updated in place
  const double* regb;      // adjoints of the face fluxes kept for flux correction (may be null)
  int leaf0, nleaf;
  int axis;
  int a0, a1, b0, b1;
  int tiles_per_leaf;
  const double* dt;
  int n_items;
};

// Remap of one new leaf from the old mesh: copy (src[0]), prolongation from
// the old leaf src[0] that is k levels coarser, or restriction from the 8 old
// children src[octant].
struct RemapEntry {
  int kind;   // 0 copy, 1 prolong, 2 restrict
  int k;
  int src[8];
};
void launch_remap(const DevMesh& neu, const DevMesh& old, const void* Uold, void* Unew, const RemapEntry* map,
                  int precision, cudaStream_t s);

// Accessors for translation units that see cello_mesh only as an opaque type.
DevMesh mesh_dev(const cello_mesh* mesh);
int mesh_precision(const cello_mesh* mesh);
cello_status set_error(cello_status status, const char* message);

// One-time kernel attribute set-up (dynamic shared memory limits), done
// outside any stream capture.
void prepare_kernels();
void prepare_kernels_f32();
void prepare_kernels_f64();

// Launchers (defined in the kernel translation units).
void launch_neighbour_table(const DevMesh& m, const unsigned long long* keys, int8_t* kind, int* idx,
                            int* fine8, cudaStream_t s);
// Ghost refresh of leaves [leaf0, leaf0+nleaf) in phases, in this order: the
// listed slow faces (leaf * 6 + face of the faces of these leaves whose
// neighbour is not a same-level leaf: their phase regions computed from leaf
// interiors), then the same-level face copies along x, y and z (each phase
// reads the margins the earlier ones filled in the face neighbours).
// `phases` selects a subset; a phase must have run on every leaf before the
// next one starts.
enum RefreshPhase : int { kRefreshSlow = 1, kRefreshX = 2, kRefreshY = 4, kRefreshZ = 8, kRefreshAll = 15 };
void launch_refresh_f32(const DevMesh& m, float* U, int leaf0, int nleaf, const int* slow, int nslow,
                        int phases, cudaStream_t s);
void launch_refresh_f64(const DevMesh& m, double* U, int leaf0, int nleaf, const int* slow, int nslow,
                        int phases, cudaStream_t s);
void launch_sweep_f32(const DevMesh& m, const SweepParams& p, int pencils, cudaStream_t s);
void launch_sweep_f64(const DevMesh& m, const SweepParams& p, int pencils, cudaStream_t s);
// Dual-energy sweeps (both float32 forms, k_de_f32.cu; float64, k_de_f64.cu),
// launched by the planners above with the grid they computed.
template <int NB, int P, int MINB>
void launch_sweep_de_f32(const DevMesh& m, const SweepParams& p, int grid, cudaStream_t s);
template <int NB, int CT, int MINB, int VEC>
void launch_stream_de_f32(const DevMesh& m, const SweepParams& p, int grid, cudaStream_t s);
template <int NB>
void launch_sweep_de_f64(const DevMesh& m, const SweepParams& p, int grid, cudaStream_t s);
void prepare_kernels_de_f32();
void prepare_kernels_de_f64();
void launch_fluxcorr(const DevMesh& m, void* U, int precision, const CoarseFace* faces,
                     const int* group_start, int ngroups, const double* reg, const double* dt,
                     cudaStream_t s);
// grid > 0: that many CTAs walk the leaves (a reduction that is to run
// alongside other kernels); 0: one CTA per leaf.  The result is the same.
void launch_reduce(const DevMesh& m, const void* U, int precision, double cfl, double* partials,
                   double* dt_next, double* totals, cudaStream_t s, int grid = 0);
// The same over leaves [leaf0, leaf0 + nleaf): partials of those leaves at
// their own offsets, the min and the sums over the range only.
void launch_reduce_range(const DevMesh& m, const void* U, int precision, double cfl, double* partials, int leaf0,
                         int nleaf, double* dt_next, double* totals, cudaStream_t s, int grid = 0);
void launch_adjoint_sweep_f32(const DevMesh& m, const AdjSweepParams& p, cudaStream_t s);
void launch_adjoint_sweep_f64(const DevMesh& m, const AdjSweepParams& p, cudaStream_t s);
void launch_adjoint_refresh(const DevMesh& m, void* lam, int precision, cudaStream_t s);
// AMR form: scatter each ghost cell's adjoint onto its sources (copies,
// restrictions, limited prolongations evaluated at the refreshed state U),
// then clear the ghost adjoints.
void launch_adjoint_refresh_scatter(const DevMesh& m, const void* U, void* lam, int precision, cudaStream_t s);
void launch_fluxcorr_adjoint(const DevMesh& m, const void* lam, int precision, const CoarseFace* faces, int nfaces,
                             double* regb, const double* dt, cudaStream_t s);
void launch_zero_ghosts(const DevMesh& m, void* lam, int precision, cudaStream_t s);
void launch_reduce_partials_f32(const DevMesh& m, const float* U, double* partials, int leaf0, int nleaf, int grid,
                                cudaStream_t s);
void launch_flags(const DevMesh& m, const void* U, int precision, int field, double tau, double tau_c,
                  int8_t* flags, cudaStream_t s);
// Multigrid Poisson solver (poisson.cu) on the M^3 grid of a uniform periodic mesh.
struct PoissonScratch;
void poisson_free(PoissonScratch* p);
cudaError_t poisson_solve(PoissonScratch** scratch, const DevMesh& m, int M, double h, const double* f_leaves,
                          double* phi_leaves, int cycles, int inner, double* resid_host, cudaStream_t s);
// Tracer particles (particles.cu): lookup of the containing leaf, and one push.
void launch_particles_locate(const DevMesh& m, const unsigned long long* keys, const double lo[3], const double hi[3],
                             const double* pos, int* leaf, long count, cudaStream_t s);
void launch_particles_push(const DevMesh& m, const unsigned long long* keys, const double lo[3], const double hi[3],
                           const void* U, int precision, double* pos, int* leaf, long count, const double* dt,
                           cudaStream_t s);
// Sharded step (k_f64.cu): interiors of the listed leaves to (pack = 1) or
// from (pack = 0) buf[count][nf][n^3]; float64 flux-register slots (per
// doubles each) to or from buf[count][per].
void launch_halo_copy(const DevMesh& m, void* U, int precision, const int* ids, long count, void* buf, int pack,
                      cudaStream_t s);
void launch_flux_copy(double* reg, const int* slots, long count, long per, double* buf, int pack, cudaStream_t s);
// Interior cells of every leaf and field from src to dst (same layout, both
// device-addressable, 16-byte aligned).
void launch_interior_copy(const DevMesh& m, const void* src, void* dst, int precision, cudaStream_t s);
// Host: counted operations of one leaf's sweep (opcount.cu), update applied.
void opcount_leaf(float* slab, int n, int g, int axis, int a0, int a1, int b0, int b1, double dtdx, double gamma,
                  int riemann, int steepen, int dual, unsigned long long counts[6]);

}  // namespace cello
