// Device construction of the 27-entry neighbour table of the leaf Blocks
// (Sec. II.B: each Block's ghost data comes from neighbouring Blocks of the
// array of octrees).  Pure integer work: every entry is found by binary
// search of the Morton keys of the sorted leaves.
#include "cello_internal.h"
#include "morton.h"

namespace cello {

// Index of the leaf whose key equals `key`, or -1.
__device__ __forceinline__ int find_key(const unsigned long long* keys, int B, unsigned long long key) {
  int lo = 0, hi = B;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (keys[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return (lo < B && keys[lo] == key) ? lo : -1;
}

__global__ void neighbour_kernel(DevMesh m, const unsigned long long* keys, int8_t* kind, int* idx, int* fine8) {
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)m.B * 27) return;
  const int b = (int)(gid / 27), e = (int)(gid % 27);
  const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
  const int4 lf = m.leaf[b];
  const int L = lf.x;
  int node[3] = {lf.y + dx, lf.z + dy, lf.w + dz};
  int8_t k = kBoundary;
  int id = -1;
  int f8[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  bool inside = true;
  for (int a = 0; a < 3; ++a) {
    const int nb = m.root[a] << L;
    if (node[a] < 0 || node[a] >= nb) {
      if (m.bc[a] == 0) node[a] = (node[a] % nb + nb) % nb;
      else inside = false;
    }
  }
  if (inside) {
    const int sh = m.max_level - L;
    const int pos = find_key(keys, m.B, morton3((unsigned)node[0] << sh, (unsigned)node[1] << sh,
                                                (unsigned)node[2] << sh));
    const int plev = pos >= 0 ? m.leaf[pos].x : -1;
    if (pos >= 0 && plev == L) {
      k = kSame;
      id = pos;
    } else if (pos >= 0 && plev > L) {
      k = kFine;
      const int s1 = sh - 1;
      for (int o = 0; o < 8; ++o) {
        const unsigned cx = 2u * node[0] + (o & 1), cy = 2u * node[1] + ((o >> 1) & 1), cz = 2u * node[2] + (o >> 2);
        const int c = find_key(keys, m.B, morton3(cx << s1, cy << s1, cz << s1));
        f8[o] = (c >= 0 && m.leaf[c].x == L + 1) ? c : -1;
      }
    } else {
      const int s1 = sh + 1;
      const int c = find_key(keys, m.B, morton3((unsigned)(node[0] >> 1) << s1, (unsigned)(node[1] >> 1) << s1,
                                                (unsigned)(node[2] >> 1) << s1));
      if (c >= 0 && m.leaf[c].x == L - 1) {
        k = kCoarse;
        id = c;
      } else {
        k = -1;  // broken balance: reported by the host
      }
    }
  }
  kind[gid] = k;
  idx[gid] = id;
  for (int o = 0; o < 8; ++o) fine8[gid * 8 + o] = f8[o];
}

void launch_neighbour_table(const DevMesh& m, const unsigned long long* keys, int8_t* kind, int* idx, int* fine8,
                            cudaStream_t s) {
  const long threads = (long)m.B * 27;
  if (threads <= 0) return;
  neighbour_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(m, keys, kind, idx, fine8);
}

}  // namespace cello
