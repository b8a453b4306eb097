// Arithmetic-throughput probe for the roofline denominators: FP64 FMA on the
// CUDA cores (DFMA), FP64 mma.sync m8n8k4 (DMMA) and FP32 FMA (FFMA), each run
// on every SM with enough independent work per thread to reach the pipe's
// throughput; then DFMA and DMMA in alternate warps of the same CTAs, whose
// combined rate tells whether the two share the FP64 units (the sum of both
// rates if not, the rate of one if they do).  Prints one JSON object.  Every
// thread writes one value to out[global thread id], so the grid covers the
// output buffer exactly.
#include <cstdio>
#include <cuda_runtime.h>

template <int CH>
__global__ void dfma_loop(double* out, int iters, double a, double b) {
  double acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = threadIdx.x * 1e-3 + c;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = fma(acc[c], a, b);
  double s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void ffma_loop(float* out, int iters, float a, float b) {
  float acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = threadIdx.x * 1e-3f + c;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = fmaf(acc[c], a, b);
  float s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void dmma_loop(double* out, int iters) {
  const double a = 1.0 + threadIdx.x * 1e-6, b = 0.999;
  double c[CH][2];
#pragma unroll
  for (int k = 0; k < CH; ++k) c[k][0] = c[k][1] = k;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < CH; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  double s = 0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += c[k][0] + c[k][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Even warps: DFMA chains (it_f rounds of 8); odd warps: DMMA chains (it_m
// rounds of 4).
__global__ void dfma_dmma_mixed(double* out, int it_f, int it_m) {
  const int warp = threadIdx.x >> 5;
  double s = 0.0;
  if ((warp & 1) == 0) {
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < it_f; ++it)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], 1.0000001, 1e-9);
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c];
  } else {
    const double a = 1.0 + threadIdx.x * 1e-6, b = 0.999;
    double c[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = k;
    for (int it = 0; it < it_m; ++it)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(c[k][0]), "+d"(c[k][1])
                     : "d"(a), "d"(b));
#pragma unroll
    for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

static float time_ms(cudaEvent_t e0, cudaEvent_t e1) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

int main() {
  int dev = 0, sms = 0, clk = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  const int threads = 256, blocks = sms * 8;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters = 4096;
  dfma_loop<8><<<blocks, threads>>>(buf, 16, 1.0000001, 1e-9);  // warm-up
  cudaEventRecord(e0);
  dfma_loop<8><<<blocks, threads>>>(buf, iters, 1.0000001, 1e-9);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  const double dfma = 2.0 * 8 * iters * (double)blocks * threads / (time_ms(e0, e1) * 1e-3) / 1e12;
  dmma_loop<4><<<blocks, threads>>>(buf, 16);
  cudaEventRecord(e0);
  dmma_loop<4><<<blocks, threads>>>(buf, iters / 4);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  const double dmma = 2.0 * 8 * 8 * 4 * 4.0 * (iters / 4) * (double)blocks * (threads / 32) /
                      (time_ms(e0, e1) * 1e-3) / 1e12;
  ffma_loop<8><<<blocks, threads>>>((float*)buf, 16, 1.0000001f, 1e-9f);
  cudaEventRecord(e0);
  ffma_loop<8><<<blocks, threads>>>((float*)buf, iters * 8, 1.0000001f, 1e-9f);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  const double ffma = 2.0 * 8 * iters * 8 * (double)blocks * threads / (time_ms(e0, e1) * 1e-3) / 1e12;
  dfma_dmma_mixed<<<blocks, threads>>>(buf, 16, 4);
  cudaEventRecord(e0);
  dfma_dmma_mixed<<<blocks, threads>>>(buf, iters, iters / 4);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  const double mixed = (2.0 * 8 * iters * (double)blocks * (threads / 2) +
                        2.0 * 8 * 8 * 4 * 4.0 * (iters / 4) * (double)blocks * (threads / 64)) /
                       (time_ms(e0, e1) * 1e-3) / 1e12;
  const cudaError_t e = cudaDeviceSynchronize();
  cudaFree(buf);
  if (e != cudaSuccess) return 1;
  printf("{\"dfma_tflops\": %.4f, \"dmma_tflops\": %.4f, \"ffma_tflops\": %.3f, \"dfma_with_dmma_tflops\": %.4f, "
         "\"sms\": %d, \"clock_mhz\": %d}\n",
         dfma, dmma, ffma, mixed, sms, clk / 1000);
  return 0;
}
