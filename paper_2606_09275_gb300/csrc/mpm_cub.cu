// Scan, radix sort and unique from CUB (header-only CCCL), used by the
// once-per-step mesh build; every call runs on the context stream.
#include <cub/cub.cuh>

#include "mpm_internal.cuh"

namespace mpm {

void cub_exclusive_sum_int(mpm_ctx* c, const int* in, int* out, int n) {
  size_t bytes = 0;
  MPM_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, c->stream));
  void* tmp = grow_bytes(c, c->cub_tmp, bytes);
  MPM_CUDA(cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, n, c->stream));
}

void cub_sort_u64(mpm_ctx* c, uint64_t* keys, uint64_t* alt, int n, int end_bit) {
  cub::DoubleBuffer<uint64_t> db(keys, alt);
  size_t bytes = 0;
  MPM_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, bytes, db, n, 0, end_bit, c->stream));
  void* tmp = grow_bytes(c, c->cub_tmp, bytes);
  MPM_CUDA(cub::DeviceRadixSort::SortKeys(tmp, bytes, db, n, 0, end_bit, c->stream));
  if (db.Current() != keys)
    MPM_CUDA(cudaMemcpyAsync(keys, db.Current(), sizeof(uint64_t) * (size_t)n,
                             cudaMemcpyDeviceToDevice, c->stream));
}

void cub_sort_pairs_int(mpm_ctx* c, const int* kin, int* kout, const int* vin, int* vout, int n,
                        int end_bit) {
  size_t bytes = 0;
  MPM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kin, kout, vin, vout, n, 0, end_bit,
                                           c->stream));
  void* tmp = grow_bytes(c, c->cub_tmp, bytes);
  MPM_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, kin, kout, vin, vout, n, 0, end_bit,
                                           c->stream));
}

int cub_unique_u64(mpm_ctx* c, const uint64_t* in, uint64_t* out, int n) {
  int* d_num = (int*)c->d_red;  // slot reused: read back right away
  size_t bytes = 0;
  MPM_CUDA(cub::DeviceSelect::Unique(nullptr, bytes, in, out, d_num, n, c->stream));
  void* tmp = grow_bytes(c, c->cub_tmp, bytes);
  MPM_CUDA(cub::DeviceSelect::Unique(tmp, bytes, in, out, d_num, n, c->stream));
  MPM_CUDA(cudaMemcpyAsync(c->h_int, d_num, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MPM_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_int[0];
}

}  // namespace mpm
