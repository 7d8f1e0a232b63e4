// Positive control of the index checks of the debug build: a kernel reads element i of a buffer
// through FXI with a stated extent n that may be smaller than the buffer, so that an index in
// [n, size) must be reported although the read itself stays inside the buffer.
#include <cuda_runtime.h>

#ifndef FX_BOUNDS_CHECK
#define FX_BOUNDS_CHECK
#endif
#include "fx_check.cuh"

struct ProbeArgs {
  unsigned* status;
  const float* buf;
  float* out;
  int n, i;
};

__global__ void probe_kernel(const ProbeArgs A) {
  if (threadIdx.x == 0 && blockIdx.x == 0) A.out[0] = A.buf[FXI(A.i, A.n)];  // the checked read
}

// status: 6 device words (zeroed by the caller); buf: device buffer of at least n and i + 1
// elements; out: one device float.  Returns the cudaError_t of the launch and synchronisation.
extern "C" int fx_probe(unsigned* status, const float* buf, float* out, int n, int i) {
  probe_kernel<<<1, 32>>>(ProbeArgs{status, buf, out, n, i});
  return (int)cudaDeviceSynchronize();
}

extern "C" unsigned fx_probe_tag(void) { return fx::fxb_file_tag(__FILE__); }
