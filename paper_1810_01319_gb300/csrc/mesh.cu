// Host side of the library: the C ABI, the array-of-octrees build from
// refinement flags (Sec. II.B), the device block table and the per-step
// launch sequence (ghost refresh -> three PPM sweeps -> flux correction ->
// CFL/totals reduction), optionally replayed from a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "cello.h"
#include "cello_internal.h"
#include "morton.h"

using namespace cello;

namespace {

thread_local std::string g_last_error;

// Fields per cell: five conserved, plus rho e with the dual-energy formalism.
int nfields(const cello_mesh_desc& d) { return d.dual_energy ? 6 : 5; }

cello_status fail(cello_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

// State pools and adjoints must start on a 256-byte boundary (the ABI's
// convention): the kernels move whole 32-byte sectors and 16-byte vectors,
// which a misaligned address would turn into a device fault.
bool misaligned(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0; }
#define CELLO_REQUIRE_ALIGNED(p) \
  do { if (misaligned(p)) return fail(CELLO_EINVAL, #p " is not 256-byte aligned"); } while (0)

#define CELLO_CUDA(call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? CELLO_ENOMEM : CELLO_ECUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

struct Node {
  int L, i, j, k;
};

inline unsigned long long pack(const Node& t) {
  return ((unsigned long long)t.L << 60) | ((unsigned long long)t.i << 40) | ((unsigned long long)t.j << 20) |
         (unsigned long long)t.k;
}

inline Node child(const Node& t, int o) {
  return Node{t.L + 1, 2 * t.i + (o & 1), 2 * t.j + ((o >> 1) & 1), 2 * t.k + (o >> 2)};
}

// Leaf set with its internal (refined) ancestors, for balance queries.
struct Tree {
  const cello_mesh_desc& d;
  std::unordered_set<unsigned long long> leaves, internal;
  explicit Tree(const cello_mesh_desc& desc) : d(desc) {}

  void index(const std::vector<Node>& ls) {
    leaves.clear();
    internal.clear();
    for (const Node& t : ls) {
      leaves.insert(pack(t));
      Node p = t;
      while (p.L > 0) {
        p = Node{p.L - 1, p.i >> 1, p.j >> 1, p.k >> 1};
        if (!internal.insert(pack(p)).second) break;
      }
    }
  }

  bool wrap(int L, int a, int& v) const {
    const int nb = d.root[a] << L;
    if (v >= 0 && v < nb) return true;
    if (d.bc[a] != CELLO_PERIODIC) return false;
    v = ((v % nb) + nb) % nb;
    return true;
  }

  // True if a leaf two or more levels finer than node t touches it: some
  // same-level neighbour node is refined and one of its children that
  // touches t is refined too.
  bool touches_deeper(const Node& t) const {
    if (t.L + 2 > d.max_level) return false;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          int v[3] = {t.i + dx, t.j + dy, t.k + dz};
          bool in = true;
          for (int a = 0; a < 3; ++a) in = in && wrap(t.L, a, v[a]);
          if (!in) continue;
          const Node nb{t.L, v[0], v[1], v[2]};
          if (!internal.count(pack(nb))) continue;
          for (int o = 0; o < 8; ++o) {
            const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
            if ((dx == 1 && ox) || (dx == -1 && !ox) || (dy == 1 && oy) || (dy == -1 && !oy) || (dz == 1 && oz) ||
                (dz == -1 && !oz))
              continue;
            if (internal.count(pack(child(nb, o)))) return true;
          }
        }
    return false;
  }
};

unsigned long long leaf_key(const cello_mesh_desc& d, const Node& t) {
  const int s = d.max_level - t.L;
  return morton3((unsigned)t.i << s, (unsigned)t.j << s, (unsigned)t.k << s);
}

}  // namespace

namespace cello {
void prepare_kernels() {
  static std::once_flag once;
  std::call_once(once, [] {
    prepare_kernels_f32();
    prepare_kernels_f64();
    prepare_kernels_de_f32();
    prepare_kernels_de_f64();
  });
  // L2 fetch granularity of this process's context on the current device, set
  // once per device: 64 bytes.  The ghost refresh reads 32-byte margin
  // sectors of 160-byte rows; with the limit left unset, misses fetched
  // 128-byte lines (phase X: 3.2x its requested sectors read from DRAM).  A
  // hint of this context only, not a device setting.
  static std::mutex mu;
  static unsigned long long done = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lock(mu);
    if (!(done >> dev & 1ull)) {
      if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 64) != cudaSuccess)
        cudaGetLastError();   // a device that does not take the hint keeps its default
      done |= 1ull << dev;
    }
  }
}
}  // namespace cello

struct GraphEntry {
  const void* U;
  const double* dt;
  int parity;
  double cfl;
  double* dt_next;
  double* totals;
  cudaGraphExec_t exec;
  bool cfl_step = false;   // a cello_hydro_step_cfl graph (dt from the start state)
};

struct cello_mesh {
  cello_mesh_desc desc{};
  int B = 0, N = 0;
  std::vector<int4> leaves;
  std::vector<unsigned long long> keys;
  std::vector<int8_t> kind;
  std::vector<int> idx, fine8, face_slot;
  std::vector<CoarseFace> cfaces;
  std::vector<int> group_start;
  int nslots = 0;
  int4* d_leaf = nullptr;
  unsigned long long* d_keys = nullptr;
  int8_t* d_kind = nullptr;
  int* d_idx = nullptr;
  int* d_fine8 = nullptr;
  int* d_face_slot = nullptr;
  CoarseFace* d_cfaces = nullptr;
  int* d_group_start = nullptr;
  double* d_reg = nullptr;
  double* d_partials = nullptr;
  int* d_slow = nullptr;           // faces the refresh computes (leaf * 6 + face): neighbour not same-level
  std::vector<int> slow_start;     // per-leaf offsets into d_slow, B + 1 entries
  int exec_mode = CELLO_EXEC_BATCHED;
  int sweep_variant[3] = {0, 0, 0};   // per sweep axis; chosen by cello_autotune or set by the caller
  unsigned* d_work = nullptr;      // work counter of the persistent sweep variants
  unsigned* d_err = nullptr;       // error word set by the reduction
  PoissonScratch* poisson = nullptr;   // multigrid levels, allocated by the first Poisson solve
  double* d_zero = nullptr;        // dt = 0, for timing sweeps without changing the state
  void* adj_scratch = nullptr;   // three states for the adjoint's forward recomputation
  size_t adj_bytes = 0;
  int* d_xlist = nullptr;        // index list of the last pack/unpack call (sharded step)
  size_t xlist_cap = 0;
  std::vector<GraphEntry> graphs;
  cudaStream_t capture_stream = nullptr;
  cudaStream_t side_stream = nullptr;          // the start-state reduction of cello_hydro_step_cfl
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;

  DevMesh dev() const {
    DevMesh m;
    m.n = desc.n;
    m.g = desc.ghosts;
    m.N = N;
    m.max_level = desc.max_level;
    for (int a = 0; a < 3; ++a) {
      m.root[a] = desc.root[a];
      m.bc[a] = desc.bc[a];
    }
    m.dx0 = (desc.hi[0] - desc.lo[0]) / (desc.root[0] * desc.n);
    m.gamma = desc.gamma;
    m.riemann = desc.riemann;
    m.steepen = desc.steepening;
    m.nf = desc.dual_energy ? 6 : 5;
    m.B = B;
    m.leaf = d_leaf;
    m.kind = d_kind;
    m.idx = d_idx;
    m.fine8 = d_fine8;
    m.face_slot = d_face_slot;
    m.err = d_err;
    return m;
  }

  void release() {
    poisson_free(poisson);
    poisson = nullptr;
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
    if (capture_stream) cudaStreamDestroy(capture_stream);
    capture_stream = nullptr;
    if (side_stream) cudaStreamDestroy(side_stream);
    side_stream = nullptr;
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
    fork_ev = join_ev = nullptr;
    if (adj_scratch) cudaFree(adj_scratch);
    adj_scratch = nullptr;
    if (d_xlist) cudaFree(d_xlist);
    d_xlist = nullptr;
    xlist_cap = 0;
    if (d_work) cudaFree(d_work);
    if (d_zero) cudaFree(d_zero);
    if (d_err) cudaFree(d_err);
    d_err = nullptr;
    d_work = nullptr;
    d_zero = nullptr;
    if (d_slow) cudaFree(d_slow);
    d_slow = nullptr;
    void* ptrs[] = {d_leaf, d_keys, d_kind, d_idx, d_fine8, d_face_slot, d_cfaces, d_group_start, d_reg, d_partials};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    d_leaf = nullptr; d_keys = nullptr; d_kind = nullptr; d_idx = nullptr; d_fine8 = nullptr;
    d_face_slot = nullptr; d_cfaces = nullptr; d_group_start = nullptr; d_reg = nullptr; d_partials = nullptr;
  }
  ~cello_mesh() { release(); }
};

namespace {

cello_status check_desc(const cello_mesh_desc* d) {
  if (!d) return fail(CELLO_EINVAL, "desc is NULL");
  if (d->n != 8 && d->n != 16 && d->n != 32) return fail(CELLO_EINVAL, "n must be 8, 16 or 32");
  if (d->ghosts != kGhosts) return fail(CELLO_EINVAL, "ghosts must be 4");
  if (d->precision != 4 && d->precision != 8) return fail(CELLO_EINVAL, "precision must be 4 or 8");
  if (d->max_level < 0 || d->max_level > 10) return fail(CELLO_EINVAL, "max_level must be in [0, 10]");
  if (!(d->gamma > 1.0)) return fail(CELLO_EINVAL, "gamma must exceed 1");
  if (d->riemann != CELLO_RIEMANN_TWO_SHOCK && d->riemann != CELLO_RIEMANN_HLLC)
    return fail(CELLO_EINVAL, "riemann must be CELLO_RIEMANN_TWO_SHOCK or CELLO_RIEMANN_HLLC");
  if (d->steepening != 0 && d->steepening != 1) return fail(CELLO_EINVAL, "steepening must be 0 or 1");
  if (d->dual_energy != 0 && d->dual_energy != 1) return fail(CELLO_EINVAL, "dual_energy must be 0 or 1");
  double ext[3];
  for (int a = 0; a < 3; ++a) {
    if (d->root[a] < 1 || d->root[a] > 1024) return fail(CELLO_EINVAL, "root blocks per axis must be in [1, 1024]");
    if (d->bc[a] != CELLO_PERIODIC && d->bc[a] != CELLO_OUTFLOW) return fail(CELLO_EINVAL, "bc must be 0 or 1");
    ext[a] = (d->hi[a] - d->lo[a]) / d->root[a];
    if (!(ext[a] > 0)) return fail(CELLO_EINVAL, "hi must exceed lo");
  }
  for (int a = 1; a < 3; ++a)
    if (std::abs(ext[a] - ext[0]) > 1e-12 * ext[0]) return fail(CELLO_EINVAL, "cells must be cubes");
  return CELLO_OK;
}

// New leaf list from the previous one and flags (see cello_octree_build).
std::vector<Node> build_leaves(const cello_mesh_desc& d, const cello_mesh* prev, const int8_t* flags) {
  std::vector<Node> cur;
  if (!prev) {
    for (int k = 0; k < d.root[2]; ++k)
      for (int j = 0; j < d.root[1]; ++j)
        for (int i = 0; i < d.root[0]; ++i) cur.push_back(Node{0, i, j, k});
    return cur;
  }
  const int B = prev->B;
  std::vector<Node> old(B);
  for (int b = 0; b < B; ++b) {
    const int4 l = prev->leaves[b];
    old[b] = Node{l.x, l.y, l.z, l.w};
  }
  std::unordered_map<unsigned long long, int> flag_of;
  std::unordered_set<unsigned long long> refine;
  for (int b = 0; b < B; ++b) {
    const int f = flags ? flags[b] : 0;
    flag_of[pack(old[b])] = f;
    if (f > 0 && old[b].L < d.max_level) refine.insert(pack(old[b]));
  }
  for (const Node& t : old) {
    if (refine.count(pack(t)))
      for (int o = 0; o < 8; ++o) cur.push_back(child(t, o));
    else
      cur.push_back(t);
  }
  Tree tree(d);
  tree.index(cur);
  // coarsening candidates: complete octets of unrefined -1 leaves
  std::unordered_map<unsigned long long, int> kids;
  for (const Node& t : old)
    if (t.L > 0) kids[pack(Node{t.L - 1, t.i >> 1, t.j >> 1, t.k >> 1})]++;
  std::vector<Node> coarsen;
  for (const auto& kv : kids) {
    if (kv.second != 8) continue;
    const unsigned long long pk = kv.first;
    const Node p{(int)(pk >> 60), (int)((pk >> 40) & 0xfffff), (int)((pk >> 20) & 0xfffff), (int)(pk & 0xfffff)};
    bool ok = true;
    for (int o = 0; o < 8 && ok; ++o) {
      const unsigned long long c = pack(child(p, o));
      auto it = flag_of.find(c);
      ok = it != flag_of.end() && it->second < 0 && !refine.count(c);
    }
    if (ok && !tree.touches_deeper(p)) coarsen.push_back(p);
  }
  if (!coarsen.empty()) {
    std::unordered_set<unsigned long long> gone;
    for (const Node& p : coarsen)
      for (int o = 0; o < 8; ++o) gone.insert(pack(child(p, o)));
    std::vector<Node> next;
    for (const Node& t : cur)
      if (!gone.count(pack(t))) next.push_back(t);
    for (const Node& p : coarsen) next.push_back(p);
    cur.swap(next);
  }
  // 2:1 balance: refine every leaf touching a leaf two levels finer
  for (;;) {
    tree.index(cur);
    std::vector<Node> next;
    bool changed = false;
    for (const Node& t : cur) {
      if (tree.touches_deeper(t)) {
        changed = true;
        for (int o = 0; o < 8; ++o) next.push_back(child(t, o));
      } else {
        next.push_back(t);
      }
    }
    cur.swap(next);
    if (!changed) break;
  }
  return cur;
}

template <typename V>
cello_status upload(V** dptr, const std::vector<V>& h) {
  if (h.empty()) return CELLO_OK;
  CELLO_CUDA(cudaMalloc((void**)dptr, h.size() * sizeof(V)));
  CELLO_CUDA(cudaMemcpy(*dptr, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
  return CELLO_OK;
}

#define CELLO_TRY(expr)               \
  do {                                \
    cello_status st_ = (expr);        \
    if (st_ != CELLO_OK) return st_;  \
  } while (0)

cello_status finish_build(cello_mesh* M) {
  const cello_mesh_desc& d = M->desc;
  const int B = M->B;
  CELLO_TRY(upload(&M->d_leaf, M->leaves));
  CELLO_TRY(upload(&M->d_keys, M->keys));
  CELLO_CUDA(cudaMalloc((void**)&M->d_kind, (size_t)B * 27));
  CELLO_CUDA(cudaMalloc((void**)&M->d_idx, (size_t)B * 27 * sizeof(int)));
  CELLO_CUDA(cudaMalloc((void**)&M->d_fine8, (size_t)B * 27 * 8 * sizeof(int)));
  DevMesh dm = M->dev();
  launch_neighbour_table(dm, M->d_keys, M->d_kind, M->d_idx, M->d_fine8, 0);
  CELLO_CUDA(cudaGetLastError());
  M->kind.resize((size_t)B * 27);
  M->idx.resize((size_t)B * 27);
  M->fine8.resize((size_t)B * 27 * 8);
  CELLO_CUDA(cudaMemcpy(M->kind.data(), M->d_kind, M->kind.size(), cudaMemcpyDeviceToHost));
  CELLO_CUDA(cudaMemcpy(M->idx.data(), M->d_idx, M->idx.size() * sizeof(int), cudaMemcpyDeviceToHost));
  CELLO_CUDA(cudaMemcpy(M->fine8.data(), M->d_fine8, M->fine8.size() * sizeof(int), cudaMemcpyDeviceToHost));
  for (int8_t k : M->kind)
    if (k < 0) return fail(CELLO_EINTERNAL, "2:1 balance violated: a neighbour is two levels coarser");
  // every child of a refined neighbour node that touches the leaf must be a
  // leaf (balance); the refresh and the slope lookups index only those
  for (int b = 0; b < B; ++b)
    for (int e = 0; e < 27; ++e) {
      if (M->kind[(size_t)b * 27 + e] != kFine) continue;
      const int dd[3] = {e % 3 - 1, (e / 3) % 3 - 1, e / 9 - 1};
      for (int o = 0; o < 8; ++o) {
        const int oo[3] = {o & 1, (o >> 1) & 1, o >> 2};
        bool touch = true;
        for (int a = 0; a < 3; ++a) touch = touch && !((dd[a] == 1 && oo[a]) || (dd[a] == -1 && !oo[a]));
        if (touch && M->fine8[((size_t)b * 27 + e) * 8 + o] < 0)
          return fail(CELLO_EINTERNAL, "2:1 balance violated: a touching neighbour is two levels finer");
      }
    }
  // flux-register slots: faces whose neighbour is finer (coarse side) or coarser (fine side)
  M->face_slot.assign((size_t)B * 6, -1);
  int ns = 0;
  for (int b = 0; b < B; ++b)
    for (int f = 0; f < 6; ++f) {
      const int k = M->kind[b * 27 + face_dir(f / 2, (f & 1) ? 1 : -1)];
      if (k == kFine || k == kCoarse) M->face_slot[b * 6 + f] = ns++;
    }
  M->nslots = ns;
  M->cfaces.clear();
  M->group_start.clear();
  for (int b = 0; b < B; ++b) {
    bool first = true;
    for (int f = 0; f < 6; ++f) {
      const int axis = f / 2, side = (f & 1) ? 1 : -1;
      const int e = b * 27 + face_dir(axis, side);
      if (M->kind[e] != kFine) continue;
      CoarseFace cf;
      cf.leaf = b;
      cf.axis = axis;
      cf.side = side;
      cf.cslot = M->face_slot[b * 6 + f];
      const int t1 = axis == 0 ? 1 : 0, t2 = axis == 2 ? 1 : 2;
      for (int o2 = 0; o2 < 2; ++o2)
        for (int o1 = 0; o1 < 2; ++o1) {
          int o[3];
          o[axis] = side < 0 ? 1 : 0;
          o[t1] = o1;
          o[t2] = o2;
          const int c = M->fine8[(size_t)e * 8 + o[2] * 4 + o[1] * 2 + o[0]];
          if (c < 0) return fail(CELLO_EINTERNAL, "refined neighbour face without leaf children");
          const int fs = M->face_slot[c * 6 + 2 * axis + (side < 0 ? 1 : 0)];
          if (fs < 0) return fail(CELLO_EINTERNAL, "fine face without a register slot");
          cf.fslot[o2 * 2 + o1] = fs;
        }
      if (first) M->group_start.push_back((int)M->cfaces.size());
      first = false;
      M->cfaces.push_back(cf);
    }
  }
  if (!M->cfaces.empty()) M->group_start.push_back((int)M->cfaces.size());
  CELLO_TRY(upload(&M->d_face_slot, M->face_slot));
  CELLO_TRY(upload(&M->d_cfaces, M->cfaces));
  CELLO_TRY(upload(&M->d_group_start, M->group_start));
  if (ns > 0) CELLO_CUDA(cudaMalloc((void**)&M->d_reg, (size_t)ns * nfields(d) * d.n * d.n * sizeof(double)));
  CELLO_CUDA(cudaMalloc((void**)&M->d_partials, (size_t)std::max(B, 1) * 6 * sizeof(double)));
  // faces whose phase region the refresh computes instead of copying: those
  // whose neighbour is not a same-level leaf (coarser, finer, boundary)
  {
    std::vector<int> slow;
    M->slow_start.assign((size_t)B + 1, 0);
    for (int b = 0; b < B; ++b) {
      for (int f = 0; f < 6; ++f)
        if (M->kind[(size_t)b * 27 + face_dir(f >> 1, (f & 1) ? 1 : -1)] != kSame) slow.push_back(b * 6 + f);
      M->slow_start[b + 1] = (int)slow.size();
    }
    CELLO_TRY(upload(&M->d_slow, slow));
  }
  CELLO_CUDA(cudaMalloc((void**)&M->d_work, sizeof(unsigned)));
  CELLO_CUDA(cudaMalloc((void**)&M->d_err, sizeof(unsigned)));
  CELLO_CUDA(cudaMemset(M->d_err, 0, sizeof(unsigned)));
  CELLO_CUDA(cudaMalloc((void**)&M->d_zero, sizeof(double)));
  CELLO_CUDA(cudaMemset(M->d_zero, 0, sizeof(double)));
  CELLO_CUDA(cudaDeviceSynchronize());
  return CELLO_OK;
}

void launch_refresh(const cello_mesh* M, const DevMesh& dm, void* U, int leaf0, int nleaf, cudaStream_t s,
                    int phases = kRefreshAll) {
  const int s0 = M->slow_start[leaf0], s1 = M->slow_start[leaf0 + nleaf];
  const int* slow = M->d_slow ? M->d_slow + s0 : nullptr;
  if (M->desc.precision == 4) launch_refresh_f32(dm, static_cast<float*>(U), leaf0, nleaf, slow, s1 - s0, phases, s);
  else launch_refresh_f64(dm, static_cast<double*>(U), leaf0, nleaf, slow, s1 - s0, phases, s);
}

// Transverse pencil ranges of a sweep along `axis`: a transverse axis already
// swept this step needs interior rows only, one not yet swept all N rows.
void sweep_ranges(const cello_mesh* M, int axis, const bool swept[3], int& a0, int& a1, int& b0, int& b1) {
  const int n = M->desc.n, g = M->desc.ghosts, N = M->N;
  const int ta = axis == 2 ? 1 : 2;   // transverse A: z, or y for the z sweep
  const int tb = axis == 0 ? 1 : 0;   // transverse B: y for the x sweep, else x
  a0 = swept[ta] ? g : 0;
  a1 = swept[ta] ? g + n : N;
  b0 = swept[tb] ? g : 0;
  b1 = swept[tb] ? g + n : N;
}

// The launch sequence of one step on stream s.
// The three split sweeps of leaves [leaf0, leaf0 + nleaf) (x, y, z on even
// cycles, z, y, x on odd ones), face fluxes of coarse-fine faces into the
// registers; plain: one launch per leaf and sweep; ev (nullable): events
// after each sweep at ev[2 ..].
void enqueue_sweeps(const cello_mesh* M, const DevMesh& dm, void* U, const double* dt, int cycle, int leaf0,
                    int nleaf, bool plain, cudaStream_t s, cudaEvent_t* ev) {
  const cello_mesh_desc& d = M->desc;
  const int order[3] = {cycle % 2 == 0 ? 0 : 2, 1, cycle % 2 == 0 ? 2 : 0};
  bool swept[3] = {false, false, false};
  for (int oi = 0; oi < 3; ++oi) {
    const int axis = order[oi];
    SweepParams p{};
    p.U = U;
    p.axis = axis;
    sweep_ranges(M, axis, swept, p.a0, p.a1, p.b0, p.b1);
    const int pencils = (p.a1 - p.a0) * (p.b1 - p.b0);
    p.dt = dt;
    p.reg = M->d_reg;
    p.work = M->d_work;
    p.variant = M->sweep_variant[axis];
    if (plain) {
      for (int b = leaf0; b < leaf0 + nleaf; ++b) {
        p.leaf0 = b;
        p.nleaf = 1;
        if (d.precision == 4) launch_sweep_f32(dm, p, pencils, s);
        else launch_sweep_f64(dm, p, pencils, s);
      }
    } else if (nleaf > 0) {
      p.leaf0 = leaf0;
      p.nleaf = nleaf;
      if (d.precision == 4) launch_sweep_f32(dm, p, pencils, s);
      else launch_sweep_f64(dm, p, pencils, s);
    }
    swept[axis] = true;
    if (ev) cudaEventRecord(ev[2 + oi], s);
  }
}

void enqueue_step(const cello_mesh* M, void* U, const double* dt, int cycle, double cfl, double* dt_next,
                  double* totals, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  const cello_mesh_desc& d = M->desc;
  const DevMesh dm = M->dev();
  const int B = M->B;
  const bool plain = M->exec_mode == CELLO_EXEC_PLAIN && !ev;
  if (ev) cudaEventRecord(ev[0], s);
  if (plain)   // one launch per leaf and phase; each phase over every leaf before the next
    for (int ph : {kRefreshSlow, kRefreshX, kRefreshY, kRefreshZ})
      for (int b = 0; b < B; ++b) launch_refresh(M, dm, U, b, 1, s, ph);
  else
    launch_refresh(M, dm, U, 0, B, s);
  if (ev) cudaEventRecord(ev[1], s);
  enqueue_sweeps(M, dm, U, dt, cycle, 0, B, plain, s, ev);
  if (!M->cfaces.empty())
    launch_fluxcorr(dm, U, d.precision, M->d_cfaces, M->d_group_start, (int)M->group_start.size() - 1, M->d_reg,
                    dt, s);
  if (ev) cudaEventRecord(ev[5], s);
  if (dt_next || totals || ev) launch_reduce(dm, U, d.precision, cfl, M->d_partials, dt_next, totals, s);
  if (ev) cudaEventRecord(ev[6], s);
}

// One step whose dt is the CFL step of its start state: the reduction of the
// start state (interiors only) on the side stream while the ghost refresh
// (ghosts only) runs on s; the sweeps wait for both.
constexpr int kSideReduceCtasPerSm = 2;

void enqueue_step_cfl(const cello_mesh* M, void* U, int cycle, double cfl, double* dt_used, double* totals,
                      cudaStream_t s) {
  const cello_mesh_desc& d = M->desc;
  const DevMesh dm = M->dev();
  cudaEventRecord(M->fork_ev, s);
  cudaStreamWaitEvent(M->side_stream, M->fork_ev, 0);
  // a few resident CTAs per SM walk the leaves, so that the reduction shares
  // the SMs with the refresh's kernels (latency-bound, DRAM not saturated)
  // instead of queueing behind them
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  launch_reduce(dm, U, d.precision, cfl, M->d_partials, dt_used, totals, M->side_stream, kSideReduceCtasPerSm * sms);
  cudaEventRecord(M->join_ev, M->side_stream);
  launch_refresh(M, dm, U, 0, M->B, s);
  cudaStreamWaitEvent(s, M->join_ev, 0);
  enqueue_sweeps(M, dm, U, dt_used, cycle, 0, M->B, false, s, nullptr);
  if (!M->cfaces.empty())
    launch_fluxcorr(dm, U, d.precision, M->d_cfaces, M->d_group_start, (int)M->group_start.size() - 1, M->d_reg,
                    dt_used, s);
}

cello_status adjoint_step(cello_mesh* M, const void* Un, void* lam, const double* dt, int cycle, cudaStream_t s) {
  const cello_mesh_desc& d = M->desc;
  bool uniform_periodic = true;   // then the ghost copy's transpose is a deterministic gather
  for (int a = 0; a < 3; ++a) uniform_periodic = uniform_periodic && d.bc[a] == CELLO_PERIODIC;
  for (int b = 1; b < M->B && uniform_periodic; ++b) uniform_periodic = M->leaves[b].x == M->leaves[0].x;
  const size_t state = (size_t)M->B * nfields(d) * M->N * M->N * M->N * d.precision;
  const size_t regs = (size_t)M->nslots * nfields(d) * d.n * d.n * sizeof(double);
  if (M->adj_bytes < 3 * state + regs) {
    if (M->adj_scratch) cudaFree(M->adj_scratch);
    M->adj_scratch = nullptr;
    M->adj_bytes = 0;
    CELLO_CUDA(cudaMalloc(&M->adj_scratch, 3 * state + regs));
    M->adj_bytes = 3 * state + regs;
  }
  char* S0 = static_cast<char*>(M->adj_scratch);
  char* S1 = S0 + state;
  char* S2 = S1 + state;
  const DevMesh dm = M->dev();
  const int B = M->B;
  // forward recomputation: refreshed start state, then the states entering
  // the second and third sweeps
  CELLO_CUDA(cudaMemcpyAsync(S0, Un, state, cudaMemcpyDeviceToDevice, s));
  launch_refresh(M, dm, S0, 0, B, s);
  const int order[3] = {cycle % 2 == 0 ? 0 : 2, 1, cycle % 2 == 0 ? 2 : 0};
  char* entry[3] = {S0, S1, S2};
  bool swept[3] = {false, false, false};
  int rng[3][4];
  for (int oi = 0; oi < 3; ++oi) {
    const int axis = order[oi];
    sweep_ranges(M, axis, swept, rng[oi][0], rng[oi][1], rng[oi][2], rng[oi][3]);
    if (oi < 2) {
      CELLO_CUDA(cudaMemcpyAsync(entry[oi + 1], entry[oi], state, cudaMemcpyDeviceToDevice, s));
      SweepParams p{};
      p.U = entry[oi + 1];
      p.axis = axis;
      p.a0 = rng[oi][0]; p.a1 = rng[oi][1]; p.b0 = rng[oi][2]; p.b1 = rng[oi][3];
      const int pencils = (p.a1 - p.a0) * (p.b1 - p.b0);
      p.dt = dt;
      p.reg = nullptr;
      p.work = M->d_work;
      p.variant = M->sweep_variant[axis];
      p.leaf0 = 0;
      p.nleaf = B;
      if (d.precision == 4) launch_sweep_f32(dm, p, pencils, s);
      else launch_sweep_f64(dm, p, pencils, s);
    }
    swept[axis] = true;
  }
  // reverse: the adjoint of U_{n+1} lives on interior cells only; the
  // coarse-fine flux correction's adjoint gives the face-flux adjoints
  launch_zero_ghosts(dm, lam, d.precision, s);
  double* regb = nullptr;
  if (!M->cfaces.empty()) {
    regb = reinterpret_cast<double*>(S2 + state);
    launch_fluxcorr_adjoint(dm, lam, d.precision, M->d_cfaces, (int)M->cfaces.size(), regb, dt, s);
  }
  for (int oi = 2; oi >= 0; --oi) {
    AdjSweepParams p{};
    p.U = entry[oi];
    p.lam = lam;
    p.regb = regb;
    p.axis = order[oi];
    p.a0 = rng[oi][0]; p.a1 = rng[oi][1]; p.b0 = rng[oi][2]; p.b1 = rng[oi][3];
    const int pencils = (p.a1 - p.a0) * (p.b1 - p.b0);
    p.tiles_per_leaf = (pencils + kAdjPencils - 1) / kAdjPencils;
    p.dt = dt;
    p.leaf0 = 0;
    p.nleaf = B;
    p.n_items = B * p.tiles_per_leaf;
    if (d.precision == 4) launch_adjoint_sweep_f32(dm, p, s);
    else launch_adjoint_sweep_f64(dm, p, s);
  }
  if (uniform_periodic) launch_adjoint_refresh(dm, lam, d.precision, s);
  else launch_adjoint_refresh_scatter(dm, S0, lam, d.precision, s);
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

}  // namespace

namespace cello {
DevMesh mesh_dev(const cello_mesh* mesh) { return mesh->dev(); }
int mesh_precision(const cello_mesh* mesh) { return mesh->desc.precision; }
cello_status set_error(cello_status status, const char* message) { return fail(status, message); }
}  // namespace cello

// ====================================================================== ABI
extern "C" {

const char* cello_last_error(void) { return g_last_error.c_str(); }

cello_status cello_octree_build(const cello_mesh_desc* desc, const cello_mesh* prev, const int8_t* flags_host,
                                cello_mesh** out) {
  if (!out) return fail(CELLO_EINVAL, "out is NULL");
  *out = nullptr;
  CELLO_TRY(check_desc(desc));
  if (prev && std::memcmp(&prev->desc, desc, sizeof(cello_mesh_desc)) != 0)
    return fail(CELLO_EINVAL, "prev was built from a different description");
  prepare_kernels();
  auto* M = new (std::nothrow) cello_mesh();
  if (!M) return fail(CELLO_ENOMEM, "host allocation failed");
  M->desc = *desc;
  M->N = desc->n + 2 * desc->ghosts;
  std::vector<Node> ls = build_leaves(*desc, prev, flags_host);
  std::vector<std::pair<unsigned long long, Node>> keyed;
  keyed.reserve(ls.size());
  for (const Node& t : ls) keyed.emplace_back(leaf_key(*desc, t), t);
  std::sort(keyed.begin(), keyed.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  M->B = (int)keyed.size();
  for (const auto& kv : keyed) {
    M->keys.push_back(kv.first);
    M->leaves.push_back(make_int4(kv.second.L, kv.second.i, kv.second.j, kv.second.k));
  }
  cello_status st = finish_build(M);
  if (st != CELLO_OK) {
    delete M;
    return st;
  }
  *out = M;
  return CELLO_OK;
}

cello_status cello_mesh_from_leaves(const cello_mesh_desc* desc, const int32_t* leaves_host, int64_t count,
                                   cello_mesh** out) {
  if (!out || !leaves_host || count <= 0) return fail(CELLO_EINVAL, "NULL argument or empty leaf list");
  *out = nullptr;
  CELLO_TRY(check_desc(desc));
  std::vector<Node> ls((size_t)count);
  std::unordered_set<unsigned long long> seen;
  double volume = 0.0;
  for (int64_t b = 0; b < count; ++b) {
    const Node t{leaves_host[4 * b], leaves_host[4 * b + 1], leaves_host[4 * b + 2], leaves_host[4 * b + 3]};
    if (t.L < 0 || t.L > desc->max_level) return fail(CELLO_EINVAL, "leaf level out of range");
    const int p[3] = {t.i, t.j, t.k};
    for (int a = 0; a < 3; ++a)
      if (p[a] < 0 || p[a] >= (desc->root[a] << t.L)) return fail(CELLO_EINVAL, "leaf index out of range");
    if (!seen.insert(pack(t)).second) return fail(CELLO_EINVAL, "duplicate leaf");
    ls[(size_t)b] = t;
    volume += std::ldexp(1.0, -3 * t.L);
  }
  for (const Node& t : ls) {   // no leaf may contain another
    Node q = t;
    while (q.L > 0) {
      q = Node{q.L - 1, q.i >> 1, q.j >> 1, q.k >> 1};
      if (seen.count(pack(q))) return fail(CELLO_EINVAL, "leaves overlap");
    }
  }
  if (volume != (double)desc->root[0] * desc->root[1] * desc->root[2])
    return fail(CELLO_EINVAL, "leaves do not tile the domain");
  prepare_kernels();
  auto* M = new (std::nothrow) cello_mesh();
  if (!M) return fail(CELLO_ENOMEM, "host allocation failed");
  M->desc = *desc;
  M->N = desc->n + 2 * desc->ghosts;
  std::vector<std::pair<unsigned long long, Node>> keyed;
  for (const Node& t : ls) keyed.emplace_back(leaf_key(*desc, t), t);
  std::sort(keyed.begin(), keyed.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  M->B = (int)keyed.size();
  for (const auto& kv : keyed) {
    M->keys.push_back(kv.first);
    M->leaves.push_back(make_int4(kv.second.L, kv.second.i, kv.second.j, kv.second.k));
  }
  cello_status st = finish_build(M);
  if (st != CELLO_OK) {
    delete M;
    return st;
  }
  *out = M;
  return CELLO_OK;
}

cello_status cello_check(cello_mesh* M, uint32_t* word) {
  if (!M) return fail(CELLO_EINVAL, "mesh is NULL");
  unsigned w = 0;
  CELLO_CUDA(cudaMemcpy(&w, M->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CELLO_CUDA(cudaMemset(M->d_err, 0, sizeof(unsigned)));
  if (word) *word = w;
  if (w & 1u) return fail(CELLO_ENONFINITE, "a reduction saw a non-finite value or a non-positive density or pressure");
  return CELLO_OK;
}

void cello_mesh_free(cello_mesh* mesh) { delete mesh; }

cello_status cello_mesh_info(const cello_mesh* M, int64_t* n_leaves, int64_t* leaf_elems, int64_t* n_cf) {
  if (!M) return fail(CELLO_EINVAL, "mesh is NULL");
  if (n_leaves) *n_leaves = M->B;
  if (leaf_elems) *leaf_elems = (int64_t)nfields(M->desc) * M->N * M->N * M->N;
  if (n_cf) *n_cf = (int64_t)M->cfaces.size();
  return CELLO_OK;
}

cello_status cello_mesh_leaves(const cello_mesh* M, int32_t* out) {
  if (!M || !out) return fail(CELLO_EINVAL, "NULL argument");
  for (int b = 0; b < M->B; ++b) {
    out[4 * b] = M->leaves[b].x;
    out[4 * b + 1] = M->leaves[b].y;
    out[4 * b + 2] = M->leaves[b].z;
    out[4 * b + 3] = M->leaves[b].w;
  }
  return CELLO_OK;
}

cello_status cello_neighbour_table(const cello_mesh* M, int8_t* kind, int32_t* idx, int32_t* fine8) {
  if (!M) return fail(CELLO_EINVAL, "mesh is NULL");
  if (kind) std::memcpy(kind, M->kind.data(), M->kind.size());
  if (idx) std::memcpy(idx, M->idx.data(), M->idx.size() * sizeof(int));
  if (fine8) std::memcpy(fine8, M->fine8.data(), M->fine8.size() * sizeof(int));
  return CELLO_OK;
}

cello_status cello_refine_flags(cello_mesh* M, const void* U, int field, double tau, double tau_c, int8_t* flags,
                                void* stream) {
  if (!M || !U || !flags) return fail(CELLO_EINVAL, "NULL argument");
  if (field != 0 && field != 4) return fail(CELLO_EINVAL, "field must be 0 (density) or 4 (pressure)");
  CELLO_REQUIRE_ALIGNED(U);
  launch_flags(M->dev(), U, M->desc.precision, field, tau, tau_c, flags, (cudaStream_t)stream);
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

cello_status cello_ghost_refresh(cello_mesh* M, void* U, void* stream) {
  if (!M || !U) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(U);
  launch_refresh(M, M->dev(), U, 0, M->B, (cudaStream_t)stream);
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

cello_status cello_reduce(cello_mesh* M, const void* U, double cfl, double* dt_next, double* totals, void* stream) {
  if (!M || !U) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(U);
  launch_reduce(M->dev(), U, M->desc.precision, cfl, M->d_partials, dt_next, totals, (cudaStream_t)stream);
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

// ------------------------------------------------------------- sharded step
namespace {

// The host index list copied to the mesh's device list (grown when needed),
// on the caller's stream.
cello_status upload_list(cello_mesh* M, const std::vector<int>& h, cudaStream_t s) {
  if (h.empty()) return CELLO_OK;
  if (M->xlist_cap < h.size()) {
    if (M->d_xlist) cudaFree(M->d_xlist);
    M->d_xlist = nullptr;
    M->xlist_cap = 0;
    CELLO_CUDA(cudaMalloc((void**)&M->d_xlist, h.size() * sizeof(int)));
    M->xlist_cap = h.size();
  }
  CELLO_CUDA(cudaMemcpyAsync(M->d_xlist, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  return CELLO_OK;
}

cello_status halo_copy(cello_mesh* M, void* U, const int32_t* leaf_ids, int64_t count, void* buf, int pack,
                       void* stream) {
  if (!M || count < 0 || (count > 0 && (!U || !leaf_ids || !buf))) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(U);
  if (reinterpret_cast<uintptr_t>(buf) & 31u) return fail(CELLO_EINVAL, "buffer is not 32-byte aligned");
  std::vector<int> h((size_t)count);
  for (int64_t k = 0; k < count; ++k) {
    if (leaf_ids[k] < 0 || leaf_ids[k] >= M->B) return fail(CELLO_EINVAL, "leaf id out of range");
    h[k] = leaf_ids[k];
  }
  cudaStream_t s = (cudaStream_t)stream;
  CELLO_TRY(upload_list(M, h, s));
  launch_halo_copy(M->dev(), U, M->desc.precision, M->d_xlist, (long)count, buf, pack, s);
  CELLO_CUDA(cudaGetLastError());
  // the list is read by the kernel: a later call must not overwrite it before
  // the kernel has run, which the stream order guarantees for calls on one
  // stream
  return CELLO_OK;
}

cello_status flux_copy(cello_mesh* M, const int32_t* faces, int64_t count, double* buf, int pack, void* stream) {
  if (!M || count < 0 || (count > 0 && (!faces || !buf))) return fail(CELLO_EINVAL, "NULL argument");
  std::vector<int> h((size_t)count);
  for (int64_t k = 0; k < count; ++k) {
    if (faces[k] < 0 || faces[k] >= M->B * 6) return fail(CELLO_EINVAL, "face entry out of range");
    const int slot = M->face_slot[(size_t)faces[k]];
    if (slot < 0) return fail(CELLO_EINVAL, "a listed face is not on a coarse-fine face (no flux register)");
    h[k] = slot;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CELLO_TRY(upload_list(M, h, s));
  launch_flux_copy(M->d_reg, M->d_xlist, (long)count, (long)nfields(M->desc) * M->desc.n * M->desc.n, buf, pack, s);
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

cello_status check_range(const cello_mesh* M, int64_t leaf0, int64_t nleaf) {
  if (leaf0 < 0 || nleaf < 0 || leaf0 + nleaf > M->B) return fail(CELLO_EINVAL, "leaf range outside the mesh");
  return CELLO_OK;
}

}  // namespace

cello_status cello_halo_pack(cello_mesh* M, const void* U, const int32_t* leaf_ids, int64_t count, void* buf,
                             void* stream) {
  return halo_copy(M, const_cast<void*>(U), leaf_ids, count, buf, 1, stream);
}

cello_status cello_halo_unpack(cello_mesh* M, void* U, const int32_t* leaf_ids, int64_t count, const void* buf,
                               void* stream) {
  return halo_copy(M, U, leaf_ids, count, const_cast<void*>(buf), 0, stream);
}

cello_status cello_flux_pack(cello_mesh* M, const int32_t* faces, int64_t count, double* buf, void* stream) {
  return flux_copy(M, faces, count, buf, 1, stream);
}

cello_status cello_flux_unpack(cello_mesh* M, const int32_t* faces, int64_t count, const double* buf, void* stream) {
  return flux_copy(M, faces, count, const_cast<double*>(buf), 0, stream);
}

cello_status cello_hydro_step_part(cello_mesh* M, void* U, const double* dt, int cycle, int64_t leaf0, int64_t nleaf,
                                   int part, void* stream) {
  if (!M || !U || !dt) return fail(CELLO_EINVAL, "NULL argument");
  if (cycle < 0) return fail(CELLO_EINVAL, "cycle must be >= 0");
  if (part != 0 && part != 1) return fail(CELLO_EINVAL, "part must be 0 (refresh and sweeps) or 1 (flux correction)");
  CELLO_REQUIRE_ALIGNED(U);
  CELLO_TRY(check_range(M, leaf0, nleaf));
  cudaStream_t s = (cudaStream_t)stream;
  const DevMesh dm = M->dev();
  if (part == 0) {
    launch_refresh(M, dm, U, 0, M->B, s);
    enqueue_sweeps(M, dm, U, dt, cycle, (int)leaf0, (int)nleaf, false, s, nullptr);
  } else if (!M->cfaces.empty()) {
    // the groups (one per coarse leaf, in leaf order) whose leaf is in the range
    const int ng = (int)M->group_start.size() - 1;
    int g0 = 0, g1 = 0;
    while (g0 < ng && M->cfaces[M->group_start[g0]].leaf < leaf0) ++g0;
    g1 = g0;
    while (g1 < ng && M->cfaces[M->group_start[g1]].leaf < leaf0 + nleaf) ++g1;
    if (g1 > g0)
      launch_fluxcorr(dm, U, M->desc.precision, M->d_cfaces, M->d_group_start + g0, g1 - g0, M->d_reg, dt, s);
  }
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

cello_status cello_reduce_part(cello_mesh* M, const void* U, int64_t leaf0, int64_t nleaf, double* out_dev,
                               void* stream) {
  if (!M || !U || !out_dev) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(U);
  CELLO_TRY(check_range(M, leaf0, nleaf));
  if (nleaf == 0) return fail(CELLO_EINVAL, "empty leaf range");
  launch_reduce_range(M->dev(), U, M->desc.precision, 1.0, M->d_partials, (int)leaf0, (int)nleaf, out_dev,
                      out_dev + 1, (cudaStream_t)stream);
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

cello_status cello_set_exec(cello_mesh* M, int mode) {
  if (!M) return fail(CELLO_EINVAL, "mesh is NULL");
  if (mode < CELLO_EXEC_PLAIN || mode > CELLO_EXEC_GRAPH) return fail(CELLO_EINVAL, "unknown exec mode");
  M->exec_mode = mode;
  return CELLO_OK;
}

cello_status cello_hydro_step(cello_mesh* M, void* U, const double* dt, int cycle, double cfl, double* dt_next,
                              double* totals, void* stream) {
  if (!M || !U || !dt) return fail(CELLO_EINVAL, "NULL argument");
  if (cycle < 0) return fail(CELLO_EINVAL, "cycle must be >= 0");
  CELLO_REQUIRE_ALIGNED(U);
  cudaStream_t s = (cudaStream_t)stream;
  if (M->exec_mode != CELLO_EXEC_GRAPH) {
    enqueue_step(M, U, dt, cycle, cfl, dt_next, totals, s);
    CELLO_CUDA(cudaGetLastError());
    return CELLO_OK;
  }
  const int parity = cycle % 2;
  for (const GraphEntry& g : M->graphs)
    if (!g.cfl_step && g.U == U && g.dt == dt && g.parity == parity && g.cfl == cfl && g.dt_next == dt_next &&
        g.totals == totals) {
      CELLO_CUDA(cudaGraphLaunch(g.exec, s));
      return CELLO_OK;
    }
  if (!M->capture_stream) CELLO_CUDA(cudaStreamCreateWithFlags(&M->capture_stream, cudaStreamNonBlocking));
  cudaGraph_t graph;
  CELLO_CUDA(cudaStreamBeginCapture(M->capture_stream, cudaStreamCaptureModeThreadLocal));
  enqueue_step(M, U, dt, parity, cfl, dt_next, totals, M->capture_stream);
  CELLO_CUDA(cudaStreamEndCapture(M->capture_stream, &graph));
  cudaGraphExec_t exec;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CELLO_CUDA(e);
  if (M->graphs.size() >= 8) {
    cudaGraphExecDestroy(M->graphs.front().exec);
    M->graphs.erase(M->graphs.begin());
  }
  M->graphs.push_back(GraphEntry{U, dt, parity, cfl, dt_next, totals, exec});
  CELLO_CUDA(cudaGraphLaunch(exec, s));
  return CELLO_OK;
}

cello_status cello_hydro_step_cfl(cello_mesh* M, void* U, int cycle, double cfl, double* dt_used, double* totals,
                                  void* stream) {
  if (!M || !U || !dt_used) return fail(CELLO_EINVAL, "NULL argument");
  if (cycle < 0) return fail(CELLO_EINVAL, "cycle must be >= 0");
  CELLO_REQUIRE_ALIGNED(U);
  cudaStream_t s = (cudaStream_t)stream;
  if (!M->side_stream) CELLO_CUDA(cudaStreamCreateWithFlags(&M->side_stream, cudaStreamNonBlocking));
  if (!M->fork_ev) CELLO_CUDA(cudaEventCreateWithFlags(&M->fork_ev, cudaEventDisableTiming));
  if (!M->join_ev) CELLO_CUDA(cudaEventCreateWithFlags(&M->join_ev, cudaEventDisableTiming));
  if (M->exec_mode != CELLO_EXEC_GRAPH) {
    enqueue_step_cfl(M, U, cycle, cfl, dt_used, totals, s);
    CELLO_CUDA(cudaGetLastError());
    return CELLO_OK;
  }
  const int parity = cycle % 2;
  for (const GraphEntry& g : M->graphs)
    if (g.cfl_step && g.U == U && g.dt == dt_used && g.parity == parity && g.cfl == cfl && g.totals == totals) {
      CELLO_CUDA(cudaGraphLaunch(g.exec, s));
      return CELLO_OK;
    }
  if (!M->capture_stream) CELLO_CUDA(cudaStreamCreateWithFlags(&M->capture_stream, cudaStreamNonBlocking));
  cudaGraph_t graph;
  CELLO_CUDA(cudaStreamBeginCapture(M->capture_stream, cudaStreamCaptureModeThreadLocal));
  enqueue_step_cfl(M, U, parity, cfl, dt_used, totals, M->capture_stream);
  CELLO_CUDA(cudaStreamEndCapture(M->capture_stream, &graph));
  cudaGraphExec_t exec;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CELLO_CUDA(e);
  if (M->graphs.size() >= 8) {
    cudaGraphExecDestroy(M->graphs.front().exec);
    M->graphs.erase(M->graphs.begin());
  }
  GraphEntry ge{U, dt_used, parity, cfl, nullptr, totals, exec};
  ge.cfl_step = true;
  M->graphs.push_back(ge);
  CELLO_CUDA(cudaGraphLaunch(exec, s));
  return CELLO_OK;
}

cello_status cello_remap(const cello_mesh* old, const void* U_old, const cello_mesh* neu, void* U_new,
                         void* stream) {
  if (!old || !neu || !U_old || !U_new) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(U_old);
  CELLO_REQUIRE_ALIGNED(U_new);
  if (std::memcmp(&old->desc, &neu->desc, sizeof(cello_mesh_desc)) != 0)
    return fail(CELLO_EINVAL, "meshes built from different descriptions");
  std::unordered_map<unsigned long long, int> where;
  for (int b = 0; b < old->B; ++b) {
    const int4 l = old->leaves[b];
    where[pack(Node{l.x, l.y, l.z, l.w})] = b;
  }
  std::vector<RemapEntry> map(neu->B);
  for (int b = 0; b < neu->B; ++b) {
    const int4 l = neu->leaves[b];
    const Node t{l.x, l.y, l.z, l.w};
    RemapEntry e{};
    auto it = where.find(pack(t));
    if (it != where.end()) {
      e.kind = 0;
      e.src[0] = it->second;
    } else {
      bool found = false;
      for (int k = 1; k <= t.L && !found; ++k) {
        auto a = where.find(pack(Node{t.L - k, t.i >> k, t.j >> k, t.k >> k}));
        if (a != where.end()) {
          e.kind = 1;
          e.k = k;
          e.src[0] = a->second;
          found = true;
        }
      }
      if (!found) {
        e.kind = 2;
        for (int o = 0; o < 8; ++o) {
          auto c = where.find(pack(child(t, o)));
          if (c == where.end()) return fail(CELLO_EINVAL, "meshes are not one adaptation apart");
          e.src[o] = c->second;
        }
      }
    }
    map[b] = e;
  }
  RemapEntry* d_map = nullptr;
  CELLO_CUDA(cudaMalloc((void**)&d_map, map.size() * sizeof(RemapEntry)));
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(d_map, map.data(), map.size() * sizeof(RemapEntry), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    launch_remap(neu->dev(), old->dev(), U_old, U_new, d_map, neu->desc.precision, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the map is freed below
  cudaFree(d_map);
  CELLO_CUDA(e);
  return CELLO_OK;
}

cello_status cello_hydro_adjoint_step(cello_mesh* M, const void* Un, void* lam, const double* dt, int cycle,
                                      void* stream) {
  if (!M || !Un || !lam || !dt) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(Un);
  CELLO_REQUIRE_ALIGNED(lam);
  if (cycle < 0) return fail(CELLO_EINVAL, "cycle must be >= 0");
  if (M->desc.riemann != CELLO_RIEMANN_TWO_SHOCK || M->desc.steepening || M->desc.dual_energy)
    return fail(CELLO_EINVAL,
                "the adjoint step is written for the two-shock solver without contact steepening or dual energy");
  return adjoint_step(M, Un, lam, dt, cycle, (cudaStream_t)stream);
}

cello_status cello_set_sweep_variants(cello_mesh* M, const int* variants) {
  if (!M || !variants) return fail(CELLO_EINVAL, "NULL argument");
  const int nv = M->desc.precision == 4 ? sweep_variant_count_f32() : sweep_variant_count_f64();
  for (int a = 0; a < 3; ++a)
    if (variants[a] < 0 || variants[a] >= nv) return fail(CELLO_EINVAL, "sweep variant out of range");
  for (int a = 0; a < 3; ++a) M->sweep_variant[a] = variants[a];
  for (auto& g : M->graphs) cudaGraphExecDestroy(g.exec);
  M->graphs.clear();
  return CELLO_OK;
}

cello_status cello_set_sweep_variant(cello_mesh* M, int variant) {
  const int v[3] = {variant, variant, variant};
  return cello_set_sweep_variants(M, v);
}

cello_status cello_autotune(cello_mesh* M, void* U, int* variants_out, float* ms_out, int ms_len, void* stream) {
  if (!M || !U) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(U);
  cudaStream_t s = (cudaStream_t)stream;
  const cello_mesh_desc& d = M->desc;
  const DevMesh dm = M->dev();
  const int nv = d.precision == 4 ? sweep_variant_count_f32() : sweep_variant_count_f64();
  const int nleaf = std::min(M->B, 4096);   // per-leaf cost is uniform: a sample of leaves suffices
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) CELLO_CUDA(cudaEventCreate(&ev[i]));
  int best[3] = {0, 0, 0};
  float best_ms[3] = {1e30f, 1e30f, 1e30f};
  cudaError_t err = cudaSuccess;
  for (int v = 0; v < nv && err == cudaSuccess; ++v) {
    float vbest[3] = {1e30f, 1e30f, 1e30f};
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
      float axis_ms[3] = {0, 0, 0};
      // the sweeps of an even (x, y, z) and an odd (z, y, x) cycle, dt = 0 (state unchanged):
      // each axis is timed in both of its positions
      for (int parity = 0; parity < 2 && err == cudaSuccess; ++parity) {
        const int order[3] = {parity == 0 ? 0 : 2, 1, parity == 0 ? 2 : 0};
        bool swept[3] = {false, false, false};
        cudaEventRecord(ev[0], s);
        for (int oi = 0; oi < 3; ++oi) {
          const int axis = order[oi];
          SweepParams p{};
          p.U = U;
          p.axis = axis;
          sweep_ranges(M, axis, swept, p.a0, p.a1, p.b0, p.b1);
          const int pencils = (p.a1 - p.a0) * (p.b1 - p.b0);
          p.dt = M->d_zero;
          p.reg = nullptr;
          p.work = M->d_work;
          p.variant = v;
          p.leaf0 = 0;
          p.nleaf = nleaf;
          if (d.precision == 4) launch_sweep_f32(dm, p, pencils, s);
          else launch_sweep_f64(dm, p, pencils, s);
          swept[axis] = true;
          cudaEventRecord(ev[oi + 1], s);
        }
        err = cudaEventSynchronize(ev[3]);
        for (int oi = 0; oi < 3 && err == cudaSuccess; ++oi) {
          float ms = 0;
          err = cudaEventElapsedTime(&ms, ev[oi], ev[oi + 1]);
          axis_ms[order[oi]] += ms;
        }
      }
      if (rep > 0)   // the first repetition warms up
        for (int a = 0; a < 3; ++a) vbest[a] = std::min(vbest[a], axis_ms[a]);
    }
    for (int a = 0; a < 3; ++a) {
      if (ms_out && 3 * v + a < ms_len) ms_out[3 * v + a] = vbest[a];
      if (vbest[a] < best_ms[a]) {
        best_ms[a] = vbest[a];
        best[a] = v;
      }
    }
  }
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  CELLO_CUDA(err);
  CELLO_CUDA(cudaGetLastError());
  if (variants_out)
    for (int a = 0; a < 3; ++a) variants_out[a] = best[a];
  return cello_set_sweep_variants(M, best);
}

cello_status cello_hydro_step_host(cello_mesh* M, void* U_host, void* U_dev, double dt_host, double* dt_dev,
                                   int cycle, double cfl, double* scratch_dev, double* out_host, void* stream) {
  if (!M || !U_host || !U_dev || !dt_dev || !scratch_dev || !out_host) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(U_dev);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)M->B * nfields(M->desc) * M->N * M->N * M->N * (size_t)M->desc.precision;
  // Host memory with a device address (page-locked, or any host memory where
  // the GPU reads the host's page tables), 16-byte aligned: the SMs read and
  // write its interior cells only (the step rewrites every ghost cell from
  // interiors before reading one).  Otherwise whole-buffer copies.
  void* h_dev = nullptr;
  bool mapped = false;
  if ((reinterpret_cast<uintptr_t>(U_host) & 15u) == 0) {
    if (cudaHostGetDevicePointer(&h_dev, U_host, 0) == cudaSuccess) mapped = h_dev != nullptr;
    else cudaGetLastError();   // no device address for this memory
  }
  const DevMesh dm = M->dev();
  if (mapped) launch_interior_copy(dm, h_dev, U_dev, M->desc.precision, s);
  else CELLO_CUDA(cudaMemcpyAsync(U_dev, U_host, bytes, cudaMemcpyHostToDevice, s));
  CELLO_CUDA(cudaMemcpyAsync(dt_dev, &dt_host, sizeof(double), cudaMemcpyHostToDevice, s));
  CELLO_TRY(cello_hydro_step(M, U_dev, dt_dev, cycle, cfl, scratch_dev, scratch_dev + 1, stream));
  if (mapped) launch_interior_copy(dm, U_dev, h_dev, M->desc.precision, s);
  else CELLO_CUDA(cudaMemcpyAsync(U_host, U_dev, bytes, cudaMemcpyDeviceToHost, s));
  CELLO_CUDA(cudaMemcpyAsync(out_host, scratch_dev, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CELLO_CUDA(cudaStreamSynchronize(s));
  return CELLO_OK;
}

cello_status cello_particles_locate(cello_mesh* M, const double* pos, int32_t* leaf, int64_t count, void* stream) {
  if (!M || (count > 0 && (!pos || !leaf)) || count < 0) return fail(CELLO_EINVAL, "NULL argument or negative count");
  launch_particles_locate(M->dev(), M->d_keys, M->desc.lo, M->desc.hi, pos, leaf, (long)count, (cudaStream_t)stream);
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

cello_status cello_particles_push(cello_mesh* M, const void* U, double* pos, int32_t* leaf, int64_t count,
                                  const double* dt, void* stream) {
  if (!M || !U || !dt || (count > 0 && (!pos || !leaf)) || count < 0)
    return fail(CELLO_EINVAL, "NULL argument or negative count");
  CELLO_REQUIRE_ALIGNED(U);
  launch_particles_push(M->dev(), M->d_keys, M->desc.lo, M->desc.hi, U, M->desc.precision, pos, leaf, (long)count, dt,
                        (cudaStream_t)stream);
  CELLO_CUDA(cudaGetLastError());
  return CELLO_OK;
}

cello_status cello_poisson_solve(cello_mesh* M, const double* f, double* phi, int cycles, int inner,
                                 double* resid_host, void* stream) {
  if (!M || !f || !phi || cycles < 1) return fail(CELLO_EINVAL, "NULL argument or cycles < 1");
  if (inner != 4 && inner != 8) return fail(CELLO_EINVAL, "inner precision must be 4 or 8");
  const cello_mesh_desc& d = M->desc;
  for (int a = 0; a < 3; ++a)
    if (d.bc[a] != CELLO_PERIODIC || d.root[a] != d.root[0])
      return fail(CELLO_EINVAL, "the Poisson solver needs a cubic root array, periodic on every axis");
  const int L = M->leaves[0].x;
  for (const int4& lf : M->leaves)
    if (lf.x != L) return fail(CELLO_EINVAL, "the Poisson solver needs a uniform mesh (every leaf at one level)");
  const long Mg = (long)d.root[0] * (1L << L) * d.n;
  if (Mg / d.n > 512) return fail(CELLO_EINVAL, "grid too large for the Poisson solver (more than 512 blocks per axis)");
  const double h = std::ldexp((d.hi[0] - d.lo[0]) / (d.root[0] * d.n), -L);
  CELLO_CUDA(poisson_solve(&M->poisson, M->dev(), (int)Mg, h, f, phi, cycles, inner, resid_host,
                           (cudaStream_t)stream));
  return CELLO_OK;
}

cello_status cello_sweep_opcount(const cello_mesh* M, float* U_host, const int32_t* leaf_ids, int64_t count,
                                 double dt, int cycle, double* out) {
  if (!M || !U_host || !leaf_ids || !out || count <= 0) return fail(CELLO_EINVAL, "NULL argument or empty sample");
  if (M->desc.precision != 4) return fail(CELLO_EINVAL, "operation counts are taken on float32 meshes");
  for (int64_t i = 0; i < count; ++i)
    if (leaf_ids[i] < 0 || leaf_ids[i] >= M->B) return fail(CELLO_EINVAL, "leaf id out of range");
  const cello_mesh_desc& d = M->desc;
  const long slab = (long)nfields(d) * M->N * M->N * M->N;
  const double dx0 = (d.hi[0] - d.lo[0]) / (d.root[0] * d.n);
  for (int k = 0; k < 3 * 8; ++k) out[k] = 0.0;
  const int order[3] = {cycle % 2 == 0 ? 0 : 2, 1, cycle % 2 == 0 ? 2 : 0};
  bool swept[3] = {false, false, false};
  for (int oi = 0; oi < 3; ++oi) {
    const int axis = order[oi];
    int a0, a1, b0, b1;
    sweep_ranges(M, axis, swept, a0, a1, b0, b1);
    unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < count; ++i) {
      const double dtdx = dt / std::ldexp(dx0, -M->leaves[leaf_ids[i]].x);
      opcount_leaf(U_host + i * slab, d.n, d.ghosts, axis, a0, a1, b0, b1, dtdx, d.gamma, d.riemann, d.steepening,
                   d.dual_energy, c);
    }
    for (int k = 0; k < 6; ++k) out[oi * 8 + k] = (double)c[k];
    out[oi * 8 + 6] = (double)count * (a1 - a0) * (b1 - b0);
    out[oi * 8 + 7] = out[oi * 8 + 6] * d.n;
    swept[axis] = true;
  }
  return CELLO_OK;
}

cello_status cello_profile_step(cello_mesh* M, void* U, const double* dt, int cycle, double cfl, float* phase_ms,
                                void* stream) {
  if (!M || !U || !dt || !phase_ms) return fail(CELLO_EINVAL, "NULL argument");
  CELLO_REQUIRE_ALIGNED(U);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev[7];
  for (int i = 0; i < 7; ++i) CELLO_CUDA(cudaEventCreate(&ev[i]));
  enqueue_step(M, U, dt, cycle, cfl, nullptr, nullptr, s, ev);
  cudaError_t e = cudaEventSynchronize(ev[6]);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&phase_ms[i], ev[i], ev[i + 1]);
  for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
  CELLO_CUDA(e);
  return CELLO_OK;
}

}  // extern "C"
