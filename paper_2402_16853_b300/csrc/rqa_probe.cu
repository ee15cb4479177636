// rqa_probe.cu -- rqa_probe_alu(): measured FP32 issue throughput of the
// operations the distance loop uses, for the roofline's denominator.  Every
// thread of a full-occupancy grid runs eight independent dependency chains
// of one operation; ops/s counts one operation per lane for the scalar
// forms and two for the packed f32x2 forms.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rqa.h"

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long pk(float a, float b) {
  unsigned long long r;
  asm volatile("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}

template <int KIND>
__global__ void alu_probe_kernel(float* out, int iters, float s) {
  float a[kChains];
  unsigned long long p[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = s * (float)(threadIdx.x + c);
    p[c] = pk(a[c], a[c] + 1.0f);
  }
  const float b = 0.999999f, d = 1e-7f;
  const unsigned long long pb = pk(b, b), pd = pk(d, d);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (KIND == 0) {
        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(b), "f"(d));
      } else if (KIND == 1) {
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(pb), "l"(pd));
      } else if (KIND == 2) {
        asm volatile("add.rn.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(d));
      } else if (KIND == 3) {
        asm volatile("sub.rn.f32x2 %0, %0, %1;" : "+l"(p[c]) : "l"(pd));
      } else {
        asm volatile("max.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(b));
      }
    }
  }
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p[c]));
    acc += a[c] + lo + hi;
  }
  if (acc == 12345.678f) out[0] = acc;  // keeps the chains alive
}

template <int KIND>
double run_probe(int sms, float* out, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st) {
  const int threads = 256, iters = 1 << 14;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, alu_probe_kernel<KIND>, threads, 0);
  if (per_sm < 1) per_sm = 1;
  const int blocks = per_sm * sms * 4;
  alu_probe_kernel<KIND><<<blocks, threads, 0, st>>>(out, iters / 16, 1e-3f);  // warm-up
  cudaEventRecord(e0, st);
  alu_probe_kernel<KIND><<<blocks, threads, 0, st>>>(out, iters, 1e-3f);
  cudaEventRecord(e1, st);
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const double per_instr = (KIND == 1 || KIND == 3) ? 2.0 : 1.0;
  const double ops = (double)blocks * threads * iters * kChains * per_instr;
  return ms > 0.f ? ops / (ms * 1e-3) : -1.0;
}

}  // namespace

extern "C" int rqa_probe_alu(int32_t kind, double* ops_per_s) {
  if (!ops_per_s || kind < 0 || kind > 4) return RQA_EINVAL;
  int dev = 0, sms = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RQA_ENODEV;
  }
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return RQA_ENODEV;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return RQA_ENOMEM;
  }
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double r = -1.0;
  switch (kind) {
    case 0: r = run_probe<0>(sms, out, e0, e1, st); break;
    case 1: r = run_probe<1>(sms, out, e0, e1, st); break;
    case 2: r = run_probe<2>(sms, out, e0, e1, st); break;
    case 3: r = run_probe<3>(sms, out, e0, e1, st); break;
    default: r = run_probe<4>(sms, out, e0, e1, st); break;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(out);
  if (e != cudaSuccess || r < 0.0) return RQA_ECUDA;
  *ops_per_s = r;
  return RQA_OK;
}
