// fp_addbench.cu -- the additions benchmark of Sec. 5.1 on the GPU: two sets
// of vectors over F_p added pairwise, many times over, in two storage forms:
//
//  * contiguous bytes: one symbol per byte, four per 32-bit word, added with
//    per-byte SIMD operations (add, subtract p, keep the smaller: a byte sum
//    s < 2p is reduced exactly by min(s, s - p) because s - p wraps above s
//    when s < p);
//  * bit-sliced natural encoding: r slices of 32-bit words hold 32 symbols,
//    added with the exact bit-sliced formulas (Alg. 3 for p = 3, Alg. 4 for
//    p = 7, ripple add and conditional subtract otherwise).
//
// The repetitions form a dependent chain, c <- c + b starting from c = a, so
// every repetition is computed and the result is a + reps * b (mod p), which
// a plain mod-p computation checks.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/fpcode.h"
#include "../../include/fpcode_testing.h"
#include "fp_bitslice.cuh"
#include "fp_internal.h"

namespace {

#define AB_CUDA(call)                                                           \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess) {                                                    \
      fph::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));       \
      return FPCODE_ECUDA;                                                      \
    }                                                                           \
  } while (0)

// One thread: one word of every slice of one 32-symbol group.
template <int P, int R>
__global__ void add_sliced_kernel(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b,
                                  uint32_t *__restrict__ c, int groups, int reps, int p) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= groups) return;
  uint32_t x[R], y[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    x[i] = a[(size_t)i * groups + gi];  // slice-major: coalesced per slice
    y[i] = b[(size_t)i * groups + gi];
  }
  for (int t = 0; t < reps; ++t) {
    uint32_t s[R];
    fpbs::add_exact<P, R>(x, y, s, p);
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] = s[i];
  }
#pragma unroll
  for (int i = 0; i < R; ++i) c[(size_t)i * groups + gi] = x[i];
}

// One thread: one 32-bit word of four byte symbols.
__global__ void add_bytes_kernel(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b,
                                 uint32_t *__restrict__ c, int words, int reps, uint32_t pppp) {
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= words) return;
  uint32_t x = a[wi];
  const uint32_t y = b[wi];
  for (int t = 0; t < reps; ++t) {
    const uint32_t s = __vadd4(x, y);
    x = __vminu4(s, __vsub4(s, pppp));
  }
  c[wi] = x;
}

template <int P, int R>
int run_sliced(const std::vector<uint32_t> &ha, const std::vector<uint32_t> &hb, std::vector<uint32_t> &hc,
               int groups, int reps, int p, cudaStream_t st, double *ms) {
  uint32_t *d = nullptr;
  const size_t words = (size_t)R * groups;
  AB_CUDA(cudaMalloc(&d, 3 * words * sizeof(uint32_t)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = FPCODE_OK;
  do {
    if (cudaMemcpyAsync(d, ha.data(), words * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d + words, hb.data(), words * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = FPCODE_ECUDA;
      break;
    }
    const int threads = 256, blocks = (groups + threads - 1) / threads;
    cudaEventRecord(e0, st);
    add_sliced_kernel<P, R><<<blocks, threads, 0, st>>>(d, d + words, d + 2 * words, groups, reps, p);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hc.data(), d + 2 * words, words * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = FPCODE_ECUDA;
      break;
    }
    float f = 0;
    cudaEventElapsedTime(&f, e0, e1);
    *ms = f;
  } while (0);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (rc) fph::set_error("fpcode_bench_additions: CUDA error in the sliced run");
  return rc;
}

}  // namespace

extern "C" int fpcode_bench_additions(int p, int sliced, int nvec, int nsym, int reps, const uint8_t *a,
                                      const uint8_t *b, uint8_t *out, void *stream, double *ms) {
  if (!a || !b || !out || !ms || nvec < 1 || nsym < 1 || reps < 0 || (sliced && p != 3 && p != 7) ||
      !fph::is_odd_prime(p) || p > 127) {
    fph::set_error("fpcode_bench_additions: p in {3, 7} (sliced) or an odd prime < 128 (bytes), sizes >= 1");
    return FPCODE_EINVAL;
  }
  const size_t total = (size_t)nvec * nsym;
  for (size_t i = 0; i < total; ++i)
    if (a[i] >= p || b[i] >= p) {
      fph::set_error("fpcode_bench_additions: symbol >= p");
      return FPCODE_EINVAL;
    }
  cudaStream_t st = (cudaStream_t)stream;
  if (sliced) {
    // groups of 32 symbols along each vector; vectors padded to a multiple of 32
    const int gpv = (nsym + 31) / 32;
    const int groups = nvec * gpv;
    const int R = p == 3 ? 2 : 3;
    std::vector<uint32_t> ha((size_t)R * groups, 0), hb((size_t)R * groups, 0), hc((size_t)R * groups, 0);
    for (int v = 0; v < nvec; ++v)
      for (int s = 0; s < nsym; ++s) {
        const size_t g = (size_t)v * gpv + s / 32;
        const uint32_t bit = 1u << (s % 32);
        const uint8_t x = a[(size_t)v * nsym + s], y = b[(size_t)v * nsym + s];
        for (int i = 0; i < R; ++i) {
          if ((x >> i) & 1) ha[(size_t)i * groups + g] |= bit;
          if ((y >> i) & 1) hb[(size_t)i * groups + g] |= bit;
        }
      }
    const int rc = p == 3 ? run_sliced<3, 2>(ha, hb, hc, groups, reps, p, st, ms)
                          : run_sliced<7, 3>(ha, hb, hc, groups, reps, p, st, ms);
    if (rc) return rc;
    for (int v = 0; v < nvec; ++v)
      for (int s = 0; s < nsym; ++s) {
        const size_t g = (size_t)v * gpv + s / 32;
        uint8_t x = 0;
        for (int i = 0; i < R; ++i) x |= (uint8_t)(((hc[(size_t)i * groups + g] >> (s % 32)) & 1u) << i);
        out[(size_t)v * nsym + s] = x;
      }
    return FPCODE_OK;
  }
  // bytes: four symbols per word, padded with zeros
  const size_t words = (total + 3) / 4;
  std::vector<uint32_t> ha(words, 0), hb(words, 0), hc(words, 0);
  std::memcpy(ha.data(), a, total);
  std::memcpy(hb.data(), b, total);
  uint32_t *d = nullptr;
  AB_CUDA(cudaMalloc(&d, 3 * words * sizeof(uint32_t)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = FPCODE_OK;
  do {
    if (cudaMemcpyAsync(d, ha.data(), words * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d + words, hb.data(), words * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = FPCODE_ECUDA;
      break;
    }
    const int threads = 256, blocks = (int)((words + threads - 1) / threads);
    const uint32_t pppp = 0x01010101u * (uint32_t)p;
    cudaEventRecord(e0, st);
    add_bytes_kernel<<<blocks, threads, 0, st>>>(d, d + words, d + 2 * words, (int)words, reps, pppp);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hc.data(), d + 2 * words, words * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = FPCODE_ECUDA;
      break;
    }
    float f = 0;
    cudaEventElapsedTime(&f, e0, e1);
    *ms = f;
  } while (0);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (rc) {
    fph::set_error("fpcode_bench_additions: CUDA error in the byte run");
    return rc;
  }
  std::memcpy(out, hc.data(), total);
  return FPCODE_OK;
}
