// Throughput micro-benchmark of the arithmetic the self-join kernels can use
// on this GPU: FP64 FMA on CUDA cores (DFMA), FP64 tensor-core MMA through
// mma.sync .f64 (m8n8k4, m16n8k4, m16n8k16), FP32 FMA, and bf16 mma.sync.
// Each kernel runs independent dependency chains long enough to saturate its
// pipe; the best of 5 timed launches (CUDA events) is reported per
// configuration of blocks per SM.
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096
__global__ void dfma_k(double* out, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4=x0+4,x5=x0+5,x6=x0+6,x7=x0+7;
  for (int i = 0; i < ITERS; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4+x5+x6+x7;
}
__global__ void ffma_k(float* out, float a, float b) {
  float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4=x0+4,x5=x0+5,x6=x0+6,x7=x0+7;
  for (int i = 0; i < ITERS; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3+x4+x5+x6+x7;
}
// DFMA with every operand in a register (no constant-bank operand) and 16
// independent chains.
__global__ void dfma_reg_k(double* out, double a0, double b0) {
  const double a = a0 + 1e-17 * threadIdx.x, b = b0 * (1.0 + 1e-17 * threadIdx.x);
  double x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = threadIdx.x + k;
  for (int i = 0; i < ITERS / 2; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void dmma884_k(double* out, double av) {
  double a = av + threadIdx.x, b = av - threadIdx.x;
  double c[4][2] = {};
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[j][0]), "+d"(c[j][1]) : "d"(a), "d"(b));
  }
  double s = 0; for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void dmma1684_k(double* out, double av) {
  double a0 = av + threadIdx.x, a1 = a0 + 1, b = av - threadIdx.x;
  double c[4][4] = {};
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
                   : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3]) : "d"(a0), "d"(a1), "d"(b));
  }
  double s = 0; for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void dmma16816_k(double* out, double av) {
  double a[8], b[4];
  for (int k = 0; k < 8; ++k) a[k] = av + threadIdx.x + k;
  for (int k = 0; k < 4; ++k) b[k] = av - threadIdx.x - k;
  double c[2][4] = {};
  for (int i = 0; i < ITERS / 4; ++i) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
                   : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
                   : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                     "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
  double s = 0; for (int j = 0; j < 2; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void mmabf16_k(float* out, unsigned av) {
  unsigned a[4] = {av, av + 1, av + 2, av + 3}, b[2] = {av + 4, av + 5};
  float c[4][4] = {};
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0; for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <typename F>
float timeit(F f) {
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  f(); cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0); f(); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
  }
  return best;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("%s SMs=%d clk=%d kHz cc=%d.%d\n", p.name, p.multiProcessorCount, clk, p.major, p.minor);
  int sms = p.multiProcessorCount;
  double* dbuf; float* fbuf; cudaMalloc(&dbuf, 1 << 26); cudaMalloc(&fbuf, 1 << 26);
  for (int bpsm : {1, 2, 4, 8}) {
    int blocks = sms * bpsm, thr = 256;
    float ms = timeit([&] { dfma_k<<<blocks, thr>>>(dbuf, 1.0000001, 1e-9); });
    double flops = 2.0 * 8 * ITERS * (double)blocks * thr;
    printf("DFMA  bpsm=%d: %.3f ms  %.3f TFLOP/s  %.2f DFMA/clk/SM(@max)\n", bpsm, ms, flops / ms / 1e9,
           flops / 2 / (ms * 1e-3) / sms / (clk * 1e3));
    ms = timeit([&] { dfma_reg_k<<<blocks, thr>>>(dbuf, 1.0000001, 1e-9); });
    printf("DFMA(reg) bpsm=%d: %.3f ms  %.3f TFLOP/s  %.2f DFMA/clk/SM(@max)\n", bpsm, ms, flops / ms / 1e9,
           flops / 2 / (ms * 1e-3) / sms / (clk * 1e3));
    ms = timeit([&] { ffma_k<<<blocks, thr>>>(fbuf, 1.0000001f, 1e-9f); });
    flops = 2.0 * 8 * ITERS * (double)blocks * thr;
    printf("FFMA  bpsm=%d: %.3f ms  %.3f TFLOP/s\n", bpsm, ms, flops / ms / 1e9);
    ms = timeit([&] { dmma884_k<<<blocks, thr>>>(dbuf, 1.0); });
    flops = 2.0 * 8 * 8 * 4 * 4 * ITERS * (double)blocks * (thr / 32);
    printf("DMMA m8n8k4   bpsm=%d: %.3f ms  %.3f TFLOP/s\n", bpsm, ms, flops / ms / 1e9);
    ms = timeit([&] { dmma1684_k<<<blocks, thr>>>(dbuf, 1.0); });
    flops = 2.0 * 16 * 8 * 4 * 4 * ITERS * (double)blocks * (thr / 32);
    printf("DMMA m16n8k4  bpsm=%d: %.3f ms  %.3f TFLOP/s\n", bpsm, ms, flops / ms / 1e9);
    ms = timeit([&] { dmma16816_k<<<blocks, thr>>>(dbuf, 1.0); });
    flops = 2.0 * 16 * 8 * 16 * 2 * (ITERS / 4) * (double)blocks * (thr / 32);
    printf("DMMA m16n8k16 bpsm=%d: %.3f ms  %.3f TFLOP/s\n", bpsm, ms, flops / ms / 1e9);
    ms = timeit([&] { mmabf16_k<<<blocks, thr>>>(fbuf, 0x3f803f80u); });
    flops = 2.0 * 16 * 8 * 16 * 4 * ITERS * (double)blocks * (thr / 32);
    printf("HMMA bf16 m16n8k16 (mma.sync) bpsm=%d: %.3f ms  %.3f TFLOP/s\n", bpsm, ms, flops / ms / 1e9);
  }
  cudaError_t e = cudaGetLastError();
  printf("status: %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
