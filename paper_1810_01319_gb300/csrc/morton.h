// Morton interleave of three 21-bit block indices (x in the lowest bit of
// each triple), the sort key of the leaf Blocks.
#pragma once

#include <cuda_runtime.h>

namespace cello {

__host__ __device__ inline unsigned long long spread3(unsigned v) {
  unsigned long long x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__host__ __device__ inline unsigned long long morton3(unsigned x, unsigned y, unsigned z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

}  // namespace cello
