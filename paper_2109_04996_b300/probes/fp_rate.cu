// Arithmetic-rate probe of one GPU: instructions per clock per SM of FP32
// FMA, packed FP32x2 FMA, FP64 FMA and add, and the FP64 <-> FP32 and
// int -> FP32 conversions.  Every chain is data dependent (each step consumes
// the previous step's result), eight independent chains per thread, all
// threads resident (8 blocks of 256 per SM), so each kernel runs at the
// issue or pipe rate of its instruction.  Timed with CUDA events after
// warm-up; the rate is reported per SM at the SM clock given on the command
// line (MHz, default 2032).
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp_rate fp_rate.cu
//   ./fp_rate [sm_mhz]
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

constexpr int kIters = 4096;

__global__ void k_ffma(float *out, float a, float b) {
  float x[8];
  for (int j = 0; j < 8; j++) x[j] = threadIdx.x + j;
  for (int i = 0; i < kIters; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = fmaf(x[j], a, b);
  float s = 0;
  for (int j = 0; j < 8; j++) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__global__ void k_ffma2(float *out, float a, float b) {
  const unsigned long long A = pack2(a, a), B = pack2(b, b);
  unsigned long long x[8];
  for (int j = 0; j < 8; j++) x[j] = pack2(threadIdx.x + j, threadIdx.x - j);
  for (int i = 0; i < kIters; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = ffma2(x[j], A, B);
  unsigned long long s = 0;
  for (int j = 0; j < 8; j++) s ^= x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)(s & 0xffff);
}

__global__ void k_dfma(float *out, double a, double b) {
  double x[8];
  for (int j = 0; j < 8; j++) x[j] = threadIdx.x + j;
  for (int i = 0; i < kIters / 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = fma(x[j], a, b);
  double s = 0;
  for (int j = 0; j < 8; j++) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__global__ void k_dadd(float *out, double a) {
  double x[8];
  for (int j = 0; j < 8; j++) x[j] = threadIdx.x + j;
  for (int i = 0; i < kIters / 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] += a;
  double s = 0;
  for (int j = 0; j < 8; j++) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// FP64 -> FP32: the float's bits are added back into the double's bit
// pattern (an integer add), so every conversion waits for the previous one.
__global__ void k_d2f(float *out, double a) {
  double d[8];
  for (int j = 0; j < 8; j++) d[j] = a * (threadIdx.x + j + 1);
  for (int i = 0; i < kIters / 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const float f = __double2float_rn(d[j]);
      d[j] = __longlong_as_double(__double_as_longlong(d[j]) + (long long)(__float_as_int(f) & 1));
    }
  double s = 0;
  for (int j = 0; j < 8; j++) s += d[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// FP32 -> FP64, the same way round.
__global__ void k_f2d(float *out, float a) {
  float f[8];
  for (int j = 0; j < 8; j++) f[j] = a * (threadIdx.x + j + 1);
  for (int i = 0; i < kIters / 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const double d = (double)f[j];
      f[j] = __int_as_float(__float_as_int(f[j]) + (int)(__double_as_longlong(d) & 1));
    }
  float s = 0;
  for (int j = 0; j < 8; j++) s += f[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// int32 -> FP32.
__global__ void k_i2f(float *out, int a) {
  int v[8];
  for (int j = 0; j < 8; j++) v[j] = a * (threadIdx.x + j + 1);
  for (int i = 0; i < kIters / 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] += __float_as_int((float)v[j]) & 3;
  int s = 0;
  for (int j = 0; j < 8; j++) s += v[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

int main(int argc, char **argv) {
  const double mhz = argc > 1 ? atof(argv[1]) : 2032.0;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = nsm * 8, nt = 256;
  float *out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * nt) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double threads = (double)blocks * nt;
  auto run = [&](const char *name, auto launch, double ops_per_thread) {
    for (int w = 0; w < 3; w++) launch();
    cudaEventRecord(e0);
    for (int r = 0; r < 5; r++) launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 5;
    const double ops = threads * ops_per_thread;
    printf("%-8s %8.3f ms  %10.1f Gop/s  %7.2f per clock per SM\n", name, ms, ops / ms / 1e6,
           ops / (ms * 1e-3) / nsm / (mhz * 1e6));
  };
  run("ffma", [&] { k_ffma<<<blocks, nt>>>(out, 0.999f, 0.001f); }, 8.0 * kIters);
  run("ffma2", [&] { k_ffma2<<<blocks, nt>>>(out, 0.999f, 0.001f); }, 16.0 * kIters);
  run("dfma", [&] { k_dfma<<<blocks, nt>>>(out, 0.999, 0.001); }, 1.0 * kIters);
  run("dadd", [&] { k_dadd<<<blocks, nt>>>(out, 0.001); }, 1.0 * kIters);
  run("f64->f32", [&] { k_d2f<<<blocks, nt>>>(out, 0.37); }, 1.0 * kIters);
  run("f32->f64", [&] { k_f2d<<<blocks, nt>>>(out, 0.37f); }, 1.0 * kIters);
  run("i32->f32", [&] { k_i2f<<<blocks, nt>>>(out, 3); }, 1.0 * kIters);
  const cudaError_t e = cudaDeviceSynchronize();
  printf("status %s, %d SMs, rates at %.0f MHz\n", cudaGetErrorString(e), nsm, mhz);
  cudaFree(out);
  return e != cudaSuccess;
}
