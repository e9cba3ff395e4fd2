// Status bookkeeping kernels of the C ABI: the handle's status word (OR of per-sample status
// bits and of the MinSR flags, read by peps_last_status), sample weights from status bits, and
// the end of a MinSR step (a step with no usable result is zeroed on the device, so that the
// call needs no host round trip).
#include "peps_kernels.cuh"
#include "peps_gb300.h"

namespace peps {

// word |= OR over the Ns per-sample status words
__global__ void k_status_or(const int* __restrict__ st, int Ns, int* word) {
  int v = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += gridDim.x * blockDim.x) v |= st[i];
  v = __reduce_or_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0 && v) atomicOr(word, v);
}

cudaError_t launch_status_or(const int* st, int Ns, int* word, cudaStream_t s) {
  if (Ns <= 0) return cudaSuccess;
  const int b = (Ns + 255) / 256;
  k_status_or<<<b < 152 ? b : 152, 256, 0, s>>>(st, Ns, word);
  return cudaGetLastError();
}

// w[i] = 0 where status[i] & mask, else 1
__global__ void k_status_weights(const int* __restrict__ st, int Ns, int mask, double* w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += gridDim.x * blockDim.x)
    w[i] = (st[i] & mask) ? 0.0 : 1.0;
}

cudaError_t launch_status_weights(const int* st, int Ns, int mask, double* w, cudaStream_t s) {
  if (Ns <= 0) return cudaSuccess;
  const int b = (Ns + 255) / 256;
  k_status_weights<<<b < 1216 ? b : 1216, 256, 0, s>>>(st, Ns, mask, w);
  return cudaGetLastError();
}

// *word |= bit when *flag != 0
__global__ void k_flag_or(const int* flag, int bit, int* word) {
  if (*flag) atomicOr(word, bit);
}

cudaError_t launch_flag_or(const int* flag, int bit, int* word, cudaStream_t s) {
  k_flag_or<<<1, 1, 0, s>>>(flag, bit, word);
  return cudaGetLastError();
}

// A MinSR step whose factorisation broke down (info[0] < 0) or whose tensor-core Gram gave up
// on a pipeline wait (*gram_err != 0) has no usable dtheta: zero it (n doubles).
__global__ void k_minsr_zero(const double* info, const int* gram_err, double* dtheta, long long n) {
  const bool bad = info[0] < 0.0 || (gram_err && *gram_err);
  if (!bad) return;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    dtheta[k] = 0.0;
}

// info[0] halved for a complex handle (its real embedding repeats every eigenvalue); info[3] =
// -1 for the factorisation route; the flags into the status word.
__global__ void k_minsr_flags(double* info, const int* gram_err, int cplx, int chol, int* word) {
  if (cplx && info[0] > 0.0) info[0] *= 0.5;
  if (chol) info[3] = -1.0;
  int f = 0;
  if (info[0] < 0.0) f |= PEPS_SW_MINSR_BREAKDOWN;
  if (gram_err && *gram_err) f |= PEPS_SW_GRAM_TIMEOUT;
  if (f) atomicOr(word, f);
}

cudaError_t launch_minsr_finish(double* info, const int* gram_err, double* dtheta, long long n, int cplx, int chol,
                                int* word, cudaStream_t s) {
  const long long b = (n + 255) / 256;
  k_minsr_zero<<<(int)(b < 1024 ? (b > 0 ? b : 1) : 1024), 256, 0, s>>>(info, gram_err, dtheta, n);
  k_minsr_flags<<<1, 1, 0, s>>>(info, gram_err, cplx, chol, word);
  return cudaGetLastError();
}

}  // namespace peps
