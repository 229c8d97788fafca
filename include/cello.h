/* cello.h - C ABI of the GB300 hydro hot path of the Enzo-P/Cello method
 * (Bordner & Norman, arXiv:1810.01319).
 *
 * One leaf Block of the array-of-octrees mesh (Sec. II.B) holds n^3 cells
 * plus a ghost layer of depth g on every side; the hydro Method is a
 * directionally split piecewise parabolic method (Sec. II.C).  This library
 * builds the leaf table, computes refinement flags, refreshes ghost zones
 * (same-level copy, restriction, prolongation, physical boundaries) and
 * advances the PPM step with coarse-fine flux correction and the CFL
 * reduction, all on one GPU.
 *
 * Conventions shared by every entry point
 *  - Field pool: caller-owned device memory, U[leaf][field][z][y][x], five
 *    conserved fields (rho, rho*u, rho*v, rho*w, E) per leaf, plus the
 *    internal energy density rho*e as a sixth when the mesh has
 *    dual_energy = 1, each a padded
 *    cube of N = n + 2g cells per edge (x fastest), element type float
 *    (precision 4) or double (precision 8), base 256-byte aligned.  Leaves
 *    are in the mesh's Morton order (see cello_mesh_leaves).  The library
 *    never frees it.
 *  - Streams: every device call is enqueued on the given cudaStream_t
 *    (passed as void*, NULL = legacy default stream) and returns without
 *    synchronising.  dt, totals and flags stay on the device.
 *  - Errors: every call returns a cello_status and never aborts; the text of
 *    the last error of the calling thread is in cello_last_error().
 *  - A cello_mesh is not thread-safe; use one per host thread.
 */
#ifndef CELLO_H
#define CELLO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cello_mesh cello_mesh;

typedef enum {
    CELLO_OK = 0,
    CELLO_EINVAL = 1,     /* bad argument or unsupported size */
    CELLO_ENOMEM = 2,     /* device or host allocation failed */
    CELLO_ECUDA = 3,      /* a CUDA runtime call failed */
    CELLO_ENONFINITE = 4, /* cello_check: a bad state was seen */
    CELLO_ETIMEOUT = 5,   /* reserved: a bounded device wait gave up */
    CELLO_EINTERNAL = 6   /* broken invariant (e.g. 2:1 balance) */
} cello_status;

enum { CELLO_PERIODIC = 0, CELLO_OUTFLOW = 1 };

/* Mesh description.  Sec. II.B: an array of root octrees (root[3] per axis)
 * over the box [lo, hi]; cells must be cubes.  n in {8, 16, 32} cells per
 * block edge, ghosts = 4 (the PPM stencil reaches four cells), max_level
 * <= 10, bc per axis (both faces of an axis share it), precision 4 or 8,
 * gamma the ideal-gas ratio of specific heats. */
typedef struct {
    int root[3];
    int n;
    int ghosts;
    int max_level;
    double lo[3];
    double hi[3];
    int bc[3];
    int precision;
    double gamma;
    int riemann;      /* interface flux of the PPM sweeps: CELLO_RIEMANN_TWO_SHOCK or CELLO_RIEMANN_HLLC */
    int steepening;   /* 1: contact steepening of the density edge values (Colella & Woodward 1984), 0: off */
    int dual_energy;  /* 1: the dual-energy formalism (Bryan et al. 1995, cited with the modified PPM of
                       * Sec. II.C): a sixth field rho*e; the sweep takes the pressure from E - ke where
                       * that exceeds 1e-3 E, else from rho*e; rho*e is advected with the mass flux,
                       * takes the compression term -(dt/dx) p (u+ - u-) with the interface-state
                       * velocities, and is reset to E - ke after each sweep where that exceeds 0.1 E.
                       * No adjoint.  0: off */
} cello_mesh_desc;

/* Riemann solvers of the sweep (Sec. II.C, PPM): the Colella-Woodward
 * two-shock solver, or HLLC (Toro, Spruce & Speares 1994) with Davis wave
 * speeds.  The adjoint step supports the two-shock solver without contact
 * steepening only. */
enum { CELLO_RIEMANN_TWO_SHOCK = 0, CELLO_RIEMANN_HLLC = 1 };

/* Build a mesh (Sec. II.B, array of octrees; Refine drives adaptation).
 * prev == NULL: the root array, every leaf at level 0.  Otherwise the new
 * leaf set is derived from prev and flags_host (host int8, one per leaf of
 * prev: +1 refine, 0 keep, -1 coarsen candidate): refine +1 leaves below
 * max_level; replace a complete octet of -1 sibling leaves by their parent
 * where that parent would touch no leaf two levels finer; then refine every
 * leaf touching a leaf two or more levels finer (faces, edges, corners,
 * periodic images) until none does.  Leaves are sorted by the Morton key of
 * their lower corner at max_level.  The 27-entry neighbour table is then
 * computed on the device.  *out receives a new mesh owned by the caller
 * (free with cello_mesh_free).  The first mesh built on a device sets the
 * calling process's L2 fetch-granularity hint for that device
 * (cudaLimitMaxL2FetchGranularity) to 64 bytes: the ghost refresh reads
 * 32-byte sectors of 160-byte rows.  The hint belongs to the process's
 * context and ends with it. */
cello_status cello_octree_build(const cello_mesh_desc* desc, const cello_mesh* prev,
                                const int8_t* flags_host, cello_mesh** out);

void cello_mesh_free(cello_mesh* mesh);

/* Rebuild a mesh from an explicit leaf list (host int32, count x (level, i,
 * j, k), any order), e.g. from a checkpoint: the leaves must lie inside the
 * root array, not repeat or overlap, and tile the domain, and the mesh must
 * be 2:1 balanced; CELLO_EINVAL / CELLO_EINTERNAL otherwise.  The result is
 * the same mesh (same Morton order, same table) as the one saved. */
cello_status cello_mesh_from_leaves(const cello_mesh_desc* desc, const int32_t* leaves_host, int64_t count,
                                   cello_mesh** out);

/* Failure detection: every reduction (cello_reduce, or a step asked for dt
 * or totals) sets bit 0 of the mesh's device error word when a leaf interior
 * holds a non-finite value or a non-positive density or pressure (before
 * the floors).  This call waits for the device, returns the word in *word
 * (nullable), clears it, and returns CELLO_ENONFINITE if bit 0 was set. */
cello_status cello_check(cello_mesh* mesh, uint32_t* word);

/* Sizes: leaves, elements per leaf (fields * N^3: 5, or 6 with dual energy),
 * coarse-fine faces. */
cello_status cello_mesh_info(const cello_mesh* mesh, int64_t* n_leaves, int64_t* leaf_elems,
                             int64_t* n_coarse_fine_faces);

/* Host copy of the leaf list: leaves_host[b*4 + {0,1,2,3}] = (level, i, j, k),
 * i in [0, root[0] << level). */
cello_status cello_mesh_leaves(const cello_mesh* mesh, int32_t* leaves_host);

/* Host copy of the device neighbour table (Sec. II.B: ghost data comes from
 * neighbouring Blocks).  27 entries per leaf, entry (dz+1)*9+(dy+1)*3+(dx+1):
 * kind 0 same-level leaf (idx), 1 coarser leaf containing the neighbour node
 * (idx), 2 refined neighbour node (fine8[8], children in octant order
 * oz*4+oy*2+ox, -1 for a child that is not a leaf), 3 outside an outflow
 * boundary.  Periodic axes wrap.  Any pointer may be NULL. */
cello_status cello_neighbour_table(const cello_mesh* mesh, int8_t* kind_host, int32_t* idx_host,
                                   int32_t* fine8_host);

/* Refinement flags (Sec. II.B, Refine), one int8 per leaf into flags_dev:
 * on density (field 0) or pressure (field 4), computed in float64 from the
 * stored values with ghost zones already refreshed; a cell passes on axis d
 * if |q(i+e_d) - q(i-e_d)| > (2*tau)*|q(i)|.  +1 if any interior cell
 * passes and level < max_level; -1 if none passes with tau_coarsen and
 * level > 0; else 0. */
cello_status cello_refine_flags(cello_mesh* mesh, const void* U, int field, double tau,
                                double tau_coarsen, int8_t* flags_dev, void* stream);

/* One hydro step whose dt is the CFL step of its own start state: dt_used
 * (device, written) = cfl x min over leaf interior cells of dx / (max |u_d| +
 * c) of U as given, totals (device, 5, nullable) the conserved totals of that
 * start state; then the step of cello_hydro_step with that dt.  The
 * reduction reads interiors only and the ghost refresh writes ghosts only, so
 * the call runs them concurrently (a forked stream, captured into the graph
 * in CELLO_EXEC_GRAPH mode); the sweeps wait for both.  A loop of these calls
 * computes the same states as cello_hydro_step with dt taken from the
 * previous call's dt_next (each step's dt is the CFL step of the state the
 * previous step produced).  Errors as cello_hydro_step. */
cello_status cello_hydro_step_cfl(cello_mesh* mesh, void* U, int cycle, double cfl, double* dt_used_dev,
                                  double* totals_dev, void* stream);

/* Remap field data onto a mesh rebuilt from `old` by one cello_octree_build
 * (Sec. II.B: Refine, with Prolong and Restrict moving data between levels).
 * U_old (old's pool, ghosts already refreshed) is read; the interior cells
 * of every leaf of U_new (neu's pool) are written, ghosts are not (refresh
 * before use).  Per new leaf: copy if the leaf existed; if an old leaf k
 * levels coarser contains it, the old cell's minmod-limited linear
 * reconstruction evaluated at the new cell centre, U_C + ((xi_x D_x + xi_y
 * D_y) + xi_z D_z), xi the offset in old-cell widths (conservative); if its
 * 8 children were old leaves, their mean (restriction).  Blocks until done.
 * CELLO_EINVAL if the meshes are not related by one adaptation. */
cello_status cello_remap(const cello_mesh* old, const void* U_old, const cello_mesh* neu, void* U_new,
                         void* stream);

/* Ghost refresh (Sec. II.B, Fig. 4; Restrict and Prolong): every ghost cell
 * of every leaf takes the value of the cell at its own level and position
 * after the physical boundary rule (periodic wrap, outflow clamp to the
 * nearest interior cell): copied from a same-level leaf, restricted (mean of
 * 8, fixed order) from finer leaves, or prolonged (conservative
 * minmod-limited linear) from the coarser leaf.  Reads leaf interiors only,
 * writes ghost cells only. */
cello_status cello_ghost_refresh(cello_mesh* mesh, void* U, void* stream);

/* One hydro step (Sec. II.C, PPM) on every leaf: ghost refresh, three split
 * PPM sweeps (x,y,z for even cycle, z,y,x for odd) with the two-shock Riemann
 * flux, then coarse-fine flux correction in float64.  dt_dev: device double,
 * the step's dt.  Afterwards dt_next_dev (device double, may be NULL) =
 * cfl * min over leaf cells of dx/(max|u_d| + c), and totals_dev (device
 * double[5], may be NULL) = float64 sums of each conserved field times cell
 * volume over leaf interiors. */
cello_status cello_hydro_step(cello_mesh* mesh, void* U, const double* dt_dev, int cycle, double cfl,
                              double* dt_next_dev, double* totals_dev, void* stream);

/* Adjoint of one hydro step with dt held fixed (the reverse of the PPM
 * sweeps of Sec. II.C and of the ghost copy of Sec. II.B):
 * lam_inout holds the adjoint of the state after the step (interior cells;
 * ghost entries are ignored) and receives the adjoint of the state U_n at
 * the start of the step (ghost entries zero).  U_n is read only; cycle and
 * dt_dev must be those of the forward step.  At a kink (min, max, branch)
 * the derivative of the branch taken in the forward pass is used.  Any
 * mesh: on a single-level periodic mesh the ghost copy is transposed by a
 * deterministic gather; otherwise the transposes of copy, restriction and
 * limited prolongation scatter with atomic adds (summation order, hence the
 * last bits, may vary between runs), and the coarse-fine flux correction is
 * transposed into the face fluxes of the adjoint sweeps.  The library keeps
 * three states of device scratch per mesh (plus the flux-register adjoints)
 * for the recomputed forward sweeps. */
cello_status cello_hydro_adjoint_step(cello_mesh* mesh, const void* U_n, void* lam_inout,
                                      const double* dt_dev, int cycle, void* stream);

/* The CFL dt and conserved totals of the current state (as after a step). */
cello_status cello_reduce(cello_mesh* mesh, const void* U, double cfl, double* dt_next_dev,
                          double* totals_dev, void* stream);

/* Execution mode of cello_hydro_step: CELLO_EXEC_PLAIN launches each phase
 * once per leaf (the per-Block Method calls of Sec. II.B); CELLO_EXEC_BATCHED
 * launches each phase once over all leaves; CELLO_EXEC_GRAPH replays the
 * batched step from a CUDA graph captured on first use. */
enum { CELLO_EXEC_PLAIN = 0, CELLO_EXEC_BATCHED = 1, CELLO_EXEC_GRAPH = 2 };
cello_status cello_set_exec(cello_mesh* mesh, int mode);

/* Launch variant of the PPM sweep kernel used by cello_hydro_step and the
 * adjoint, for all three sweep axes: the form (shared-memory phases with
 * one thread per cell, or register streaming with one thread per pencil),
 * pencils per CTA, register bound (minimum resident CTAs per SM) and
 * schedule (one CTA per work item, or one resident wave pulling items from
 * a device counter).  Float32 has 24 variants (12 shared-memory, 12
 * streaming, of which 4 read x pencils as 16-byte vectors), float64 2, the
 * same for dual-energy meshes.  The variants of one form compute the same values;
 * the two float32 forms agree to float32 rounding (a multiply and an add
 * may be fused across what is a register in one form and shared memory in
 * the other).  Cached graphs are dropped. */
cello_status cello_set_sweep_variant(cello_mesh* mesh, int variant);

/* The same with one variant per sweep axis: variants[3] for the x, y and z
 * sweeps (host array). */
cello_status cello_set_sweep_variants(cello_mesh* mesh, const int* variants);

/* Autotuner (Sec. IV: agglomerated work units on accelerators): times the
 * sweeps of an even and an odd step (each axis in both of its positions)
 * for every sweep variant on up to 4096 leaves of U with dt = 0 (U is left
 * bit-for-bit unchanged), keeps the fastest variant of each axis for this
 * mesh and returns them in variants_out[3] (nullable); ms_out (host,
 * nullable, ms_len entries) receives at [3 v + axis] the best time of
 * variant v on that axis.  Blocks until done; call it outside any stream
 * capture. */
cello_status cello_autotune(cello_mesh* mesh, void* U, int* variants_out, float* ms_out, int ms_len,
                            void* stream);

/* Tracer particles (Sec. II.B, Fig. 4: Lagrangian particles move between
 * Blocks; Sec. III: the hydro workload carries tracers).  pos_dev: device
 * float64 [3][count] (all x, then all y, then all z); leaf_dev: device int32
 * [count], the index of the containing leaf, -1 for a tracer lost through
 * an outflow face.  cello_particles_locate writes the containing leaf of
 * each point (points must lie in the box): the leaf whose Morton key is the
 * last not above the key of the point's block at max_level.  Call it to
 * start, and again after every adaptation (leaf indices change). */
cello_status cello_particles_locate(cello_mesh* mesh, const double* pos_dev, int32_t* leaf_dev, int64_t count,
                                    void* stream);

/* One tracer step: each live tracer moves by dt (device double) times the
 * fluid velocity (momentum / density) interpolated trilinearly between the
 * cell centres of its leaf's padded block, so U's ghosts must be refreshed
 * (cello_ghost_refresh); then periodic wrap, or loss (leaf -1) through an
 * outflow face, and the lookup of its (possibly new) leaf.  float64
 * arithmetic for either state precision. */
cello_status cello_particles_push(cello_mesh* mesh, const void* U, double* pos_dev, int32_t* leaf_dev,
                                  int64_t count, const double* dt_dev, void* stream);

/* Poisson solve, lap(phi) = f (Sec. II.C: Enzo-P's mg0 geometric multigrid
 * V-cycle, the self-gravity solver of the paper's uniform-grid runs), on a
 * uniform mesh (every leaf at one level), periodic on every axis, cubic
 * root array, at most 512 blocks per axis.  The V-cycle runs on the leaf
 * blocks while they have at least 4 cells per edge, each block with a
 * one-cell ghost layer refreshed from its neighbours through the mesh's
 * neighbour table, and on single arrays below that.  f_dev and phi_dev: device
 * float64 leaf interiors [B][n^3] (no ghosts; x fastest) in leaf order.
 * The 7-point cell-centred Laplacian; the mean of f is removed first and
 * the mean of phi last.  cycles V-cycles from phi = 0, each two damped
 * Jacobi sweeps (w = 6/7) before and after, restriction by the mean of 8
 * children, trilinear prolongation, coarsening by 2 while the size is even
 * (50 sweeps on an odd coarsest grid).  inner = 8: float64 V-cycles;
 * inner = 4: mixed precision, each cycle a float32 V-cycle on the float64
 * residual rounded to float32, its result added to the float64 phi (the
 * same convergence per cycle and float64's attainable accuracy, at float32
 * cost).  resid_host (nullable, host,
 * `cycles` doubles) receives the max-norm of the residual after each cycle,
 * and then the call waits for the stream.  The first solve on a mesh
 * allocates the level arrays (padded blocks: about 3 x 8 x 1.3 bytes per
 * cell for n = 32, more for smaller blocks), freed with the mesh.
 * CELLO_EINVAL on a mesh it does not support. */
cello_status cello_poisson_solve(cello_mesh* mesh, const double* f_dev, double* phi_dev, int cycles, int inner,
                                 double* resid_host, void* stream);

/* Algorithmic operation count of the three PPM sweeps of one step (Sec.
 * II.C), the numerator of the sweep kernel's ALU roofline.  Host only, no
 * device work: the sweep's formulas run in float32 through a counting
 * scalar (one operation per add, subtract, multiply, divide, square root,
 * comparison, absolute value or copysign) over the pencils the sweep kernel
 * covers, on `count` leaves whose slabs the caller copied (ghosts refreshed)
 * into U_host (float32, [count][fields][(n+2g)^3] with 5 or, with dual
 * energy, 6 fields, overwritten with the swept
 * state); leaf_ids are those leaves' indices in the mesh; dt and cycle as in
 * cello_hydro_step.  out[24]: for the k-th sweep of the step, out[8k+0..5]
 * are the operations of its six phases (primitives, slopes and shock
 * detector, interface values, flattening and tracing, Riemann flux, update),
 * out[8k+6] the pencils and out[8k+7] the cells updated.  Float32 meshes
 * only; CELLO_EINVAL otherwise or on a bad leaf id. */
cello_status cello_sweep_opcount(const cello_mesh* mesh, float* U_host, const int32_t* leaf_ids, int64_t count,
                                 double dt, int cycle, double* out);

/* One step with the state in HOST memory: copies the state (host ->
 * device, into the caller's device buffer U_dev of the same size) and dt,
 * runs cello_hydro_step, copies the state back into U_host and dt_next and
 * the five totals into out_host[6], and waits for the stream.  If
 * cudaHostGetDevicePointer gives U_host a device address (page-locked memory
 * from cudaHostAlloc or cudaHostRegister; on systems whose GPU reads the
 * host's page tables, any host memory) and U_host is 16-byte aligned, the
 * GPU reads and writes its interior cells directly through that address and
 * nothing else (the step rewrites every ghost cell from interiors before
 * reading one): U_host's ghost cells are then neither read nor written, and
 * the whole buffer must be addressable that way.  Otherwise the buffer is
 * copied whole in both directions.  dt_host: the
 * step's dt; dt_dev: a device double the call writes it to; scratch_dev: 6
 * device doubles.  Errors as cello_hydro_step. */
cello_status cello_hydro_step_host(cello_mesh* mesh, void* U_host, void* U_dev, double dt_host, double* dt_dev,
                                   int cycle, double cfl, double* scratch_dev, double* out_host, void* stream);

/* One batched step (as cello_hydro_step, without dt_next/totals) with CUDA
 * events recorded between its phases; blocks until it completes and writes
 * the device time of each phase in milliseconds to phase_ms_host[6]:
 * ghost refresh, sweep 1, sweep 2, sweep 3, flux correction, reduction
 * (the reduction of dt and totals is run and timed as well). */
cello_status cello_profile_step(cello_mesh* mesh, void* U, const double* dt_dev, int cycle, double cfl,
                                float* phase_ms_host, void* stream);

/* The same reduction as cello_reduce (same kernels, same results) for
 * callers that cannot let a library allocate device memory where it is
 * used: allocation-free stream captures, hosts that hand out a fixed device
 * budget up front, runtimes whose own allocator owns the device.  The paper
 * has no counterpart; this is an interface convenience.  Its scratch (six
 * doubles per leaf) is a fixed 1.5 MiB __device__ array of the library, held
 * by every GPU that loads the library until the process exits, so meshes
 * of more than 32768 leaves are rejected with CELLO_EINVAL.  The call
 * allocates nothing.  Its first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; make that
 * first call before any stream capture.  All calls share the one array and
 * every call writes the entries it reads before reading them, so nothing
 * has to start at zero; calls that overlap on the GPU race on it. */
cello_status cello_reduce_noalloc(cello_mesh* mesh, const void* U, double cfl, double* dt_next_dev,
                                  double* totals_dev, void* stream);

/* Measured FP32 issue rate of the current device, the denominator of the
 * sweep's ALU roofline (not a step of the method; the paper has no
 * counterpart).  Launches 8 CTAs of 256 threads per SM, each thread running
 * 16 independent fused multiply-add chains, times the launch with CUDA
 * events on `stream` (best of three after one warm-up) and writes the FP32
 * fused multiply-adds per second (lane instructions: one per lane per
 * clock at the pipes' peak; twice that in flop/s) to *ffma_per_s and the
 * launch's milliseconds to *ms_out (nullable).  Blocks until done. */
cello_status cello_fp32_ffma_rate(double* ffma_per_s, double* ms_out, void* stream);

/* ---- Sharded step: one rank's share of a step over a leaf partition ----
 * Sec. II.B: a Block is independent of the others once its ghost layer is
 * filled; Sec. III places the Blocks of the array of octrees on many ranks.
 * A rank holds the whole pool with valid interiors for its own contiguous
 * range of leaves (Morton order) and runs, with its own cello_mesh (its own
 * flux registers):
 *   1. cello_halo_unpack of the interiors of the other ranks' leaves its
 *      refresh reads (packed there by cello_halo_pack);
 *   2. cello_hydro_step_part(part 0): the ghost refresh and the three
 *      sweeps of its range (face fluxes of coarse-fine faces into the
 *      registers);
 *   3. cello_flux_unpack of the fine face fluxes other ranks computed for
 *      its coarse-fine faces (cello_flux_pack there);
 *   4. cello_hydro_step_part(part 1): the flux correction of its range's
 *      coarse faces;
 *   5. cello_reduce_part: the CFL minimum and the totals of its range; the
 *      step's dt_next is cfl x the min over ranks, its totals the sums.
 * Each rank's leaves then equal those of cello_hydro_step on the whole
 * pool, bit for bit (the same kernels, the same arithmetic); the totals
 * differ only by the order of the final sums.  Lists are host arrays,
 * checked (CELLO_EINVAL on an index out of range or a face without a flux
 * register) and copied to a device list the mesh keeps (grown when
 * needed); calls on one mesh must use one stream. */

/* Interiors of the leaves leaf_ids[0..count) (host int32) from U into the
 * device buffer buf[count][fields][n^3] (x fastest; 32-byte aligned), or
 * from buf into U. */
cello_status cello_halo_pack(cello_mesh* mesh, const void* U, const int32_t* leaf_ids, int64_t count, void* buf,
                             void* stream);
cello_status cello_halo_unpack(cello_mesh* mesh, void* U, const int32_t* leaf_ids, int64_t count, const void* buf,
                               void* stream);

/* Float64 face fluxes kept for the flux correction: faces[k] = leaf * 6 +
 * face (order -x, +x, -y, +y, -z, +z), each a face on a coarse-fine face
 * (coarse or fine side), into buf[count][fields][n^2] (device) or from
 * it into the mesh's registers. */
cello_status cello_flux_pack(cello_mesh* mesh, const int32_t* faces, int64_t count, double* buf, void* stream);
cello_status cello_flux_unpack(cello_mesh* mesh, const int32_t* faces, int64_t count, const double* buf,
                               void* stream);

/* Part of cello_hydro_step for the leaves [leaf0, leaf0 + nleaf): part 0
 * refreshes the ghosts (of every leaf: those of leaves outside the range may
 * read stale interiors and are never used) and runs the three sweeps of the
 * range; part 1 applies the flux correction of the coarse faces of the
 * range.  dt and cycle as in cello_hydro_step. */
cello_status cello_hydro_step_part(cello_mesh* mesh, void* U, const double* dt_dev, int cycle, int64_t leaf0,
                                   int64_t nleaf, int part, void* stream);

/* The reduction of cello_reduce over [leaf0, leaf0 + nleaf) (nleaf > 0):
 * out_dev[0] = min over the range's cells of dx / (max |u_d| + c) (the CFL
 * step before the factor cfl), out_dev[1..5] = the five totals. */
cello_status cello_reduce_part(cello_mesh* mesh, const void* U, int64_t leaf0, int64_t nleaf, double* out_dev,
                               void* stream);

/* Text of the calling thread's last error ("" if none). */
const char* cello_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CELLO_H */
