// pipes.cu -- issue-rate probe for the instructions the hot kernels use.
//
// One kernel per instruction kind; each thread runs 8 interdependent chains
// of that instruction for ITERS iterations.  The host prints, per kind, the
// lane-operations per SM cycle (cycles from clock64 in every CTA) and the
// kernel time; run it under ncu with the pipe counters
// (sm__inst_executed_pipe_alu / _fmaheavy / _fmalite) to see which pipe each
// kind issues on.  Every store is out[blockIdx.x * blockDim.x + threadIdx.x]
// into a buffer of exactly grid * block words.
#include <cstdio>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#define ITERS 2048
__device__ __forceinline__ unsigned h2u(__half2 h) { return *reinterpret_cast<unsigned*>(&h); }
__device__ __forceinline__ __half2 u2h(unsigned u) { return *reinterpret_cast<__half2*>(&u); }
__device__ __forceinline__ float u2f(unsigned u) { return __uint_as_float(u); }
__device__ __forceinline__ unsigned f2u(float f) { return __float_as_uint(f); }

template <int OP>
__global__ void kop(unsigned* out, long long* cyc, unsigned seed) {
  unsigned a[10];
#pragma unroll
  for (int j = 0; j < 10; j++) a[j] = ((threadIdx.x + 1) * (j + seed)) & 0x3c003c00u;
  long long t0 = clock64();
  for (int it = 0; it < ITERS; it++) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
      unsigned x = a[j], y = a[j + 1], z = a[j + 2], r;
      if (OP == 0) r = __vadd2(x, y);
      else if (OP == 1) r = __vmaxs2(x, y);
      else if (OP == 2) r = __vimax3_s16x2(x, y, z);
      else if (OP == 3) r = __viaddmax_s16x2(x, y, z);
      else if (OP == 4) asm("prmt.b32 %0, %1, %2, 0x9180;" : "=r"(r) : "r"(x), "r"(y));
      else if (OP == 5) r = x ^ (y & z);
      else if (OP == 6) r = x + y + z;
      else if (OP == 7) r = x * y + z;
      else if (OP == 8) r = max((int)x, (int)y);
      else if (OP == 9) r = h2u(__hadd2(u2h(x), u2h(y)));
      else if (OP == 10) r = h2u(__hmax2(u2h(x), u2h(y)));
      else if (OP == 11) r = h2u(__hfma2(u2h(x), u2h(y), u2h(z)));
      else if (OP == 12) r = f2u(u2f(x) + u2f(y));
      else if (OP == 13) r = f2u(fmaxf(u2f(x), u2f(y)));
      else if (OP == 14) r = __funnelshift_r(x, y, 16);
      else if (OP == 15) r = __viaddmax_s32(x, y, z);
      else if (OP == 16) r = __vimax3_s32(x, y, z);
      else if (OP == 17) r = __vsub2(x, y);
      else if (OP == 18) r = (unsigned)__vimax_s16x2_relu(x, y);
      else r = x + y;
      a[j] = r;
    }
    a[8] ^= it;
  }
  long long t1 = clock64();
  unsigned acc = 0;
#pragma unroll
  for (int j = 0; j < 10; j++) acc ^= a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

static const char* names[] = {"vadd2", "vmaxs2", "vimax3_s16x2", "viaddmax_s16x2", "prmt", "lop3", "iadd3",
                              "imad", "imax32", "hadd2", "hmax2", "hfma2", "fadd", "fmax", "funnelshift",
                              "viaddmax_s32", "vimax3_s32", "vsub2", "vimax_relu", "iadd"};

template <int OP>
void run(int nsm, unsigned* d_out, long long* d_cyc) {
  const int cps = 4, threads = 256, grid = nsm * cps;
  kop<OP><<<grid, threads>>>(d_out, d_cyc, 3u);
  cudaDeviceSynchronize();
  long long h[4096];
  cudaMemcpy(h, d_cyc, grid * sizeof(long long), cudaMemcpyDeviceToHost);
  double mean = 0;
  for (int i = 0; i < grid; i++) mean += (double)h[i];
  mean /= grid;
  double ops = (double)threads * ITERS * 8 * cps;
  float ms = 0.f;
  printf("{\"op\": \"%s\", \"lane_ops_per_clk_sm\": %.1f, \"err\": \"%s\"}\n", names[OP], ops / mean,
         cudaGetErrorString(cudaGetLastError()));
  (void)ms;
}

int main() {
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  unsigned* d_out;
  long long* d_cyc;
  cudaMalloc(&d_out, sizeof(unsigned) * nsm * 4 * 256);
  cudaMalloc(&d_cyc, sizeof(long long) * nsm * 4);
  run<0>(nsm, d_out, d_cyc); run<1>(nsm, d_out, d_cyc); run<2>(nsm, d_out, d_cyc); run<3>(nsm, d_out, d_cyc);
  run<4>(nsm, d_out, d_cyc); run<5>(nsm, d_out, d_cyc); run<6>(nsm, d_out, d_cyc); run<7>(nsm, d_out, d_cyc);
  run<8>(nsm, d_out, d_cyc); run<9>(nsm, d_out, d_cyc); run<10>(nsm, d_out, d_cyc); run<11>(nsm, d_out, d_cyc);
  run<12>(nsm, d_out, d_cyc); run<13>(nsm, d_out, d_cyc); run<14>(nsm, d_out, d_cyc); run<15>(nsm, d_out, d_cyc);
  run<16>(nsm, d_out, d_cyc); run<17>(nsm, d_out, d_cyc); run<18>(nsm, d_out, d_cyc); run<19>(nsm, d_out, d_cyc);
  cudaFree(d_out);
  cudaFree(d_cyc);
  return 0;
}
