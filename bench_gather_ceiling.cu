// Ceilings of the SpMV ingredients on this GPU: streaming, random gathers, both.
//
// Standalone microbenchmark behind the roofline discussion of the bench (the
// gather ceiling that bounds the iteration kernels on the uniformly random
// n=1e6 workload).  At that workload's sizes -- 16e6 nonzeros (int32 index +
// float32 value) gathering from a 1.5e6-entry float32 vector -- it times, with
// CUDA events (10 launches after 3 warm-ups) and three grid sizes, a 1 GiB
// copy, the index/value stream alone, hashed random 4-byte gathers, and the
// stream plus the gathers x[col].  Every loop is grid-stride over its buffer.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/gather_ceiling bench_gather_ceiling.cu
//   /tmp/gather_ceiling
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__global__ void k_stream(const int* __restrict__ col, const float* __restrict__ val, long long n, float* out) {
  float s = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += val[i] * (float)col[i];
  if (s == 123.456f) out[0] = s;
}
__global__ void k_gather_hash(const float* __restrict__ x, int nx, long long n, float* out) {
  float s = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u; h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
    s += __ldg(x + (h % (unsigned)nx));
  }
  if (s == 123.456f) out[0] = s;
}
__global__ void k_gather_col(const int* __restrict__ col, const float* __restrict__ val, const float* __restrict__ x,
                             long long n, float* out) {
  float s = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += val[i] * __ldg(x + col[i]);
  if (s == 123.456f) out[0] = s;
}
// 8 independent elements per thread per step
__global__ void k_gather_col8(const int* __restrict__ col, const float* __restrict__ val, const float* __restrict__ x,
                              long long n, float* out) {
  float s = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += 8 * stride) {
    int c[8]; float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { long long e = i + k * stride; c[k] = e < n ? col[e] : 0; v[k] = e < n ? val[e] : 0.f; }
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k] * __ldg(x + c[k]);
  }
  if (s == 123.456f) out[0] = s;
}
__global__ void k_copy(const float4* __restrict__ a, float4* __restrict__ b, long long n4) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) b[i] = a[i];
}
__global__ void k_fill_col(int* col, long long n, int nx, unsigned seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u + seed; h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
    col[i] = (int)(h % (unsigned)nx);
  }
}

int main() {
  const long long n = 16000000;   // nonzeros of the primal matrix at n=1e6
  const int nx = 1500000;         // gathered vector length (n + m)
  int* col; float* val; float* x; float* out; float4 *ca, *cb;
  const long long ncopy = 1LL << 28;  // 1 GiB
  CK(cudaMalloc(&col, n * 4)); CK(cudaMalloc(&val, n * 4)); CK(cudaMalloc(&x, nx * 4)); CK(cudaMalloc(&out, 16));
  CK(cudaMalloc(&ca, ncopy * 4)); CK(cudaMalloc(&cb, ncopy * 4));
  CK(cudaMemset(val, 0, n * 4)); CK(cudaMemset(x, 0, nx * 4)); CK(cudaMemset(ca, 0, ncopy * 4));
  k_fill_col<<<1024, 256>>>(col, n, nx, 12345u);
  CK(cudaDeviceSynchronize());
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  auto timeit = [&](const char* name, double bytes, auto launch) {
    for (int w = 0; w < 3; ++w) launch();
    cudaEventRecord(e0);
    for (int r = 0; r < 10; ++r) launch();
    cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double t = ms / 10 * 1e-3;
    printf("%-28s %9.2f us  %8.1f GB/s (%s)\n", name, t * 1e6, bytes / t / 1e9, cudaGetErrorString(cudaGetLastError()));
  };
  for (int bpsm : {4, 8, 16}) {
    int grid = sms * bpsm;
    printf("--- grid %d x 256\n", grid);
    timeit("copy 1GiB (r+w)", 2.0 * ncopy * 4, [&] { k_copy<<<grid, 256>>>(ca, cb, ncopy / 4); });
    timeit("stream col+val", 8.0 * n, [&] { k_stream<<<grid, 256>>>(col, val, n, out); });
    timeit("gather hash (sectors)", 32.0 * n, [&] { k_gather_hash<<<grid, 256>>>(x, nx, n, out); });
    timeit("col+val+gather", 8.0 * n, [&] { k_gather_col<<<grid, 256>>>(col, val, x, n, out); });
    timeit("col+val+gather x8", 8.0 * n, [&] { k_gather_col8<<<grid, 256>>>(col, val, x, n, out); });
  }
  return 0;
}
