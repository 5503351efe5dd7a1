// Multi-right-hand-side tensor-core path (BF16 storage, FP32 accumulation): placeholder until the
// tensor-core kernels are added.
#include "amg_internal.cuh"

amg_status amg_internal_tc_prepare(amg_coarse*, cudaStream_t) { return AMG_ERR_UNSUPPORTED; }
void amg_internal_free_tc(amg_coarse* h) {
  cudaFree(h->Dtc);
  cudaFree(h->Rtc);
  h->Dtc = h->Rtc = nullptr;
}
amg_status amg_internal_export_stored(amg_coarse*, double2*) { return AMG_ERR_UNSUPPORTED; }
