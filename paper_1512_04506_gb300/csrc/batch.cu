// Persistent fused restrict -> coarse apply -> prolong over several lattices: placeholder.
#include "amg_internal.cuh"

amg_status amg_internal_batch(amg_coarse* const*, int, const void* const*, void* const*, const int*, cudaStream_t) {
  return AMG_ERR_UNSUPPORTED;
}
