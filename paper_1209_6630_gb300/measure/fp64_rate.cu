// Throughput of the FP64 FMA pipe (DFMA), the FP64 tensor path (mma.sync
// m8n8k4 f64) and the FP32 FMA pipe on one GPU; the FP64 roofline of the
// Gauss-Jordan and FP64 contraction kernels is derived from the DFMA rate.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_rate fp64_rate.cu && ./fp64_rate
// Every thread writes only out[blockIdx.x * blockDim.x + threadIdx.x].
#include <cstdio>
#include <cuda_runtime.h>
__global__ void dfma_loop(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4=x0+4,x5=x0+5,x6=x0+6,x7=x0+7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void ffma_loop(float* out, int iters, float a, float b) {
  float x[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = threadIdx.x * 1e-3f + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0; for (int j = 0; j < 16; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void dmma_loop(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-6, b = 0.999;
  double c[4][2];
  for (int q = 0; q < 4; ++q) { c[q][0] = 0; c[q][1] = 0; }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c[q][0]), "+d"(c[q][1]) : "d"(a), "d"(b));
    }
  }
  double s = 0; for (int q = 0; q < 4; ++q) s += c[q][0] + c[q][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  int nsm = p.multiProcessorCount;
  printf("device %s SMs %d\n", p.name, nsm);
  int threads = 256, blocks = nsm * 8;
  double* dout; cudaMalloc(&dout, sizeof(double) * blocks * threads);
  float* fout; cudaMalloc(&fout, sizeof(float) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  // DFMA
  for (int rep = 0; rep < 2; ++rep) {
    int iters = 2000;
    cudaEventRecord(e0);
    dfma_loop<<<blocks, threads>>>(dout, iters, 0.9999, 1e-3);
    cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double flop = 2.0 * 64.0 * iters * (double)blocks * threads;
    printf("DFMA: %.3f ms  %.3f TFLOP/s\n", ms, flop / ms / 1e9);
  }
  for (int rep = 0; rep < 2; ++rep) {
    int iters = 1000;
    cudaEventRecord(e0);
    dmma_loop<<<blocks, threads>>>(dout, iters);
    cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double flop = 2.0 * 8 * 8 * 4 * 32.0 * iters * (double)blocks * threads / 32.0;
    printf("DMMA m8n8k4: %.3f ms  %.3f TFLOP/s\n", ms, flop / ms / 1e9);
  }
  for (int rep = 0; rep < 2; ++rep) {
    int iters = 20000;
    cudaEventRecord(e0);
    ffma_loop<<<blocks, threads>>>(fout, iters, 0.9999f, 1e-3f);
    cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double flop = 2.0 * 64.0 * iters * (double)blocks * threads;
    printf("FFMA: %.3f ms  %.3f TFLOP/s\n", ms, flop / ms / 1e9);
  }
  cudaError_t err = cudaDeviceSynchronize();
  printf("status: %s\n", cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
