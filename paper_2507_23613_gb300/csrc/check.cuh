// Index checks of the debugging build of libmfwh.
//
// Built with -DMFWH_BOUNDS_CHECK (paper_2507_23613_gb300.build.build(bounds_check=True), which
// writes libmfwh_bc.so), every checked global or shared-memory access of the FP64 step
// kernels first tests its index against the extent of the array it addresses.  An index out
// of range is not accessed: the kernel counts it in the handle's fault record (Geom::fault),
// keeps the first one (index, extent, source line) and goes on; it never traps.
// mfwh_debug_bounds reads the record.  In the normal build MFWH_IDX is the constant true and
// costs nothing.
#pragma once

#include <cstdint>

namespace mfwh {

// The first out-of-range index a checked kernel met, and how many it met.
struct BoundsFault {
  unsigned long long count;
  long long index, extent;
  int line;
  int pad;
};

#ifdef MFWH_BOUNDS_CHECK
__device__ __forceinline__ bool idx_ok(BoundsFault* f, int64_t i, int64_t n, int line) {
  if (i >= 0 && i < n) return true;
  if (f != nullptr && atomicAdd(&f->count, 1ull) == 0ull) {
    f->index = i;
    f->extent = n;
    f->line = line;
  }
  return false;
}
#define MFWH_IDX(fault, i, n) ::mfwh::idx_ok((fault), (int64_t)(i), (int64_t)(n), __LINE__)
#else
#define MFWH_IDX(fault, i, n) true
#endif

}  // namespace mfwh
