// Issue-rate probe for the roofline denominators of the ALU-bound kernels:
// results per clock per SM of packed FP32 (FFMA2), scalar FP32 FMA, the MUFU
// approximations the P2P kernels use (lg2, rcp, ex2, rsqrt, sin) and FP64 FMA.
//
// Every thread runs 8 independent dependency chains of one instruction in
// blocks of 256 threads, 8 blocks per SM.  Each block records its SM id and
// the clock64() values at the start and end of its loop; per SM, results per
// clock = the work of the blocks that ran there / (latest end - earliest
// start), which stays correct when fewer than 8 blocks fit at once.  The
// reported rate is the median over SMs.  Prints one JSON object.  No waits,
// no shared state: the only memory writes are one float per thread and three
// words per block.
#include <algorithm>
#include <array>
#include <cstdio>
#include <map>
#include <vector>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ float lg2a(float x) { float r; asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float rcpa(float x) { float r; asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float ex2a(float x) { float r; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float rsqa(float x) { float r; asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float sina(float x) { float r; asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }

constexpr int kChains = 8;

__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

template <int OP>
__global__ void probe(float* out, long long* cyc, int iters) {
  float2 a[kChains];
  float s[kChains];
  double dd[kChains];
  for (int k = 0; k < kChains; ++k) {
    a[k] = make_float2(1.1f + 0.01f * k + threadIdx.x * 1e-4f, 0.9f + 0.01f * k);
    s[k] = 1.3f + 0.01f * k + threadIdx.x * 1e-5f;
    dd[k] = 1.1 + 0.01 * k;
  }
  const float2 c = make_float2(0.9999f, 0.9998f), d = make_float2(1e-4f, 2e-4f);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if constexpr (OP == 0) a[k] = __ffma2_rn(a[k], c, d);
      if constexpr (OP == 1) s[k] = fmaf(s[k], 0.9999f, 1e-4f);
      if constexpr (OP == 2) s[k] = lg2a(s[k]) + 1.5f;   // the add keeps the chain in range
      if constexpr (OP == 3) s[k] = rcpa(s[k]) + 1.0f;  // x -> 1/x + 1 (no rcp(rcp(x)) folding)
      if constexpr (OP == 4) s[k] = ex2a(s[k]) * 0.5f;
      if constexpr (OP == 5) s[k] = rsqa(s[k]);
      if constexpr (OP == 6) s[k] = sina(s[k]) + 1.0f;
      if constexpr (OP == 7) dd[k] = fma(dd[k], 0.9999, 1e-4);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float r = 0.f;
  for (int k = 0; k < kChains; ++k) r += a[k].x + a[k].y + s[k] + (float)dd[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
  if (threadIdx.x == 0) {
    cyc[3 * blockIdx.x] = (long long)smid();
    cyc[3 * blockIdx.x + 1] = t0;
    cyc[3 * blockIdx.x + 2] = t1;
  }
}

}  // namespace

int main() {
  int nsm = 0, clk_khz = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  const int bps = 8, th = 256, iters = 4096;
  const int blocks = nsm * bps;
  float* out = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * th * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&cyc, (size_t)blocks * 3 * sizeof(long long)) != cudaSuccess) {
    std::printf("{\"error\": \"cudaMalloc failed\"}\n");
    return 1;
  }
  std::vector<long long> h((size_t)blocks * 3);
  const char* names[] = {"ffma2_packed", "ffma", "mufu_lg2", "mufu_rcp", "mufu_ex2", "mufu_rsqrt", "mufu_sin", "dfma"};
  void (*ks[])(float*, long long*, int) = {probe<0>, probe<1>, probe<2>, probe<3>,
                                           probe<4>, probe<5>, probe<6>, probe<7>};
  const int results_per_op[] = {2, 1, 1, 1, 1, 1, 1, 1};
  std::printf("{\"sms\": %d, \"clock_mhz_attr\": %.0f", nsm, clk_khz / 1000.0);
  const double work_per_block = (double)th * iters * kChains;
  for (int o = 0; o < 8; ++o) {
    for (int rep = 0; rep < 2; ++rep) ks[o]<<<blocks, th>>>(out, cyc, iters);
    if (cudaDeviceSynchronize() != cudaSuccess) {
      std::printf(", \"error\": \"launch failed\"}\n");
      return 1;
    }
    cudaMemcpy(h.data(), cyc, h.size() * sizeof(long long), cudaMemcpyDeviceToHost);
    std::map<long long, std::array<double, 3>> per_sm;  // sm -> (blocks, first start, last end)
    for (int b = 0; b < blocks; ++b) {
      auto it = per_sm.find(h[3 * b]);
      if (it == per_sm.end()) {
        per_sm[h[3 * b]] = {1.0, (double)h[3 * b + 1], (double)h[3 * b + 2]};
      } else {
        it->second[0] += 1.0;
        it->second[1] = std::min(it->second[1], (double)h[3 * b + 1]);
        it->second[2] = std::max(it->second[2], (double)h[3 * b + 2]);
      }
    }
    std::vector<double> rates;
    for (auto& kv : per_sm) rates.push_back(kv.second[0] * work_per_block * results_per_op[o] /
                                            (kv.second[2] - kv.second[1]));
    std::sort(rates.begin(), rates.end());
    std::printf(", \"%s\": %.2f", names[o], rates[rates.size() / 2]);
  }
  std::printf("}\n");
  cudaFree(out);
  cudaFree(cyc);
  return 0;
}
