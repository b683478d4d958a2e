// int_pipes.cu -- throughput probe for the integer operations of the sweep:
// 3-input XOR (LOP3), 32x32->64 multiply (the Philox product), 32-bit
// multiply-add, 3-input add, the acceptance carry chain (sub.cc + addc), and
// whole Philox4x32-10 blocks, per SM and clock (clock64 inside the kernels).
// The lop3.b32 / iadd3 / carry lines use inline PTX on chains whose operands
// all change every iteration, so the compiler cannot fold them.  Every thread writes one word of `out`; every block one
// word of `cyc`: both are sized grid x block and grid.  Used to bound the
// sweep's roofline; not part of the library.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define N_ITER 4096
__global__ void k_lop3(uint32_t* out, uint32_t seed, long long* cyc) {
  uint32_t a[8]; for (int i=0;i<8;++i) a[i]=seed+threadIdx.x*8+i;
  long long c0 = clock64();
  for (int it=0; it<N_ITER; ++it) {
    #pragma unroll
    for (int i=0;i<8;++i) a[i] = a[i] ^ (a[(i+1)&7] + 0) ^ (uint32_t)it;  // xor3
  }
  long long c1 = clock64();
  uint32_t s=0; for (int i=0;i<8;++i) s^=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
  if (threadIdx.x==0) cyc[blockIdx.x]=c1-c0;
}
__global__ void k_lop3_ptx(uint32_t* out, uint32_t seed, long long* cyc) {
  uint32_t a[8]; for (int i=0;i<8;++i) a[i]=seed*(i+1)+threadIdx.x*8+i;
  long long c0 = clock64();
  for (int it=0; it<N_ITER; ++it) {
    #pragma unroll
    for (int i=0;i<8;++i) {
      uint32_t r;
      asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a[i]), "r"(a[(i+1)&7]), "r"(a[(i+5)&7]));
      a[i] = r;
    }
  }
  long long c1 = clock64();
  uint32_t s=0; for (int i=0;i<8;++i) s^=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
  if (threadIdx.x==0) cyc[blockIdx.x]=c1-c0;
}
__global__ void k_iadd3(uint32_t* out, uint32_t seed, long long* cyc) {
  uint32_t a[8]; for (int i=0;i<8;++i) a[i]=seed*(i+1)+threadIdx.x*8+i;
  long long c0 = clock64();
  for (int it=0; it<N_ITER; ++it) {
    #pragma unroll
    for (int i=0;i<8;++i) {
      uint32_t r;
      asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(a[i]), "r"(a[(i+1)&7]));
      a[i] = r ^ (uint32_t)it;
    }
  }
  long long c1 = clock64();
  uint32_t s=0; for (int i=0;i<8;++i) s^=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
  if (threadIdx.x==0) cyc[blockIdx.x]=c1-c0;
}
// the acceptance step of the sweep: acc = 2 acc + [r >= t] (two instructions)
__global__ void k_carry(uint32_t* out, uint32_t seed, long long* cyc) {
  uint32_t a[8], acc[8]; for (int i=0;i<8;++i) { a[i]=seed*(i+1)+threadIdx.x*8+i; acc[i]=0; }
  long long c0 = clock64();
  for (int it=0; it<N_ITER; ++it) {
    #pragma unroll
    for (int i=0;i<8;++i) {
      uint32_t d, o;
      asm volatile("sub.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %4;" : "=r"(d), "=r"(o) : "r"(a[i]), "r"(a[(i+3)&7]), "r"(acc[i]));
      acc[i] = o;
      a[i] = d;
    }
  }
  long long c1 = clock64();
  uint32_t s=0; for (int i=0;i<8;++i) s^=a[i]^acc[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
  if (threadIdx.x==0) cyc[blockIdx.x]=c1-c0;
}
__global__ void k_mulwide(uint32_t* out, uint32_t seed, long long* cyc) {
  uint32_t a[8]; for (int i=0;i<8;++i) a[i]=seed+threadIdx.x*8+i;
  long long c0 = clock64();
  for (int it=0; it<N_ITER; ++it) {
    #pragma unroll
    for (int i=0;i<8;++i) { uint64_t p = (uint64_t)0xD2511F53u * a[i]; a[i] = (uint32_t)(p>>32) + (uint32_t)p; }
  }
  long long c1 = clock64();
  uint32_t s=0; for (int i=0;i<8;++i) s^=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
  if (threadIdx.x==0) cyc[blockIdx.x]=c1-c0;
}
__global__ void k_imad(uint32_t* out, uint32_t seed, long long* cyc) {
  uint32_t a[8]; for (int i=0;i<8;++i) a[i]=seed+threadIdx.x*8+i;
  long long c0 = clock64();
  for (int it=0; it<N_ITER; ++it) {
    #pragma unroll
    for (int i=0;i<8;++i) a[i] = a[i] * 0xD2511F53u + a[(i+3)&7];
  }
  long long c1 = clock64();
  uint32_t s=0; for (int i=0;i<8;++i) s^=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
  if (threadIdx.x==0) cyc[blockIdx.x]=c1-c0;
}
__global__ void k_philox(uint32_t* out, uint32_t seed, long long* cyc) {
  uint32_t c0=threadIdx.x+blockIdx.x*blockDim.x, c1=seed, c2=7, c3=1, acc=0;
  long long t0 = clock64();
  for (int it=0; it<N_ITER/16; ++it) {
    uint32_t x0=c0+it, x1=c1, x2=c2, x3=c3, k0=seed, k1=seed*3;
    #pragma unroll
    for (int r=0;r<10;++r){ uint32_t ka=k0+r*0x9E3779B9u, kb=k1+r*0xBB67AE85u;
      uint32_t ha=__umulhi(0xD2511F53u,x0), la=0xD2511F53u*x0, hb=__umulhi(0xCD9E8D57u,x2), lb=0xCD9E8D57u*x2;
      x0=hb^x1^ka; x1=lb; x2=ha^x3^kb; x3=la; }
    acc ^= x0 ^ x1 ^ x2 ^ x3;
  }
  long long t1 = clock64();
  out[blockIdx.x*blockDim.x+threadIdx.x]=acc;
  if (threadIdx.x==0) cyc[blockIdx.x]=t1-t0;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int threads=256, blocks=sms*8;
  uint32_t* out; long long* cyc; cudaMalloc(&out, blocks*threads*4); cudaMalloc(&cyc, blocks*8);
  long long* h = new long long[blocks];
  struct K { const char* name; void (*f)(uint32_t*,uint32_t,long long*); double ops_per_thread; } ks[] = {
    {"lop3(xor3)", k_lop3, 8.0*N_ITER}, {"lop3.b32 (ptx)", k_lop3_ptx, 8.0*N_ITER},
    {"add.u32 (+xor)", k_iadd3, 16.0*N_ITER}, {"sub.cc+addc pair", k_carry, 8.0*N_ITER},
    {"imad.wide(mulhi+mullo)", k_mulwide, 8.0*N_ITER},
    {"imad", k_imad, 8.0*N_ITER}, {"philox blocks", k_philox, (double)(N_ITER/16)} };
  for (auto& k : ks) {
    for (int rep=0; rep<2; ++rep) {
      cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
      cudaEventRecord(e0); k.f<<<blocks,threads>>>(out, 123, cyc); cudaEventRecord(e1); cudaEventSynchronize(e1);
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      cudaMemcpy(h, cyc, blocks*8, cudaMemcpyDeviceToHost);
      double avgc=0; for (int i=0;i<blocks;++i) avgc+=h[i]; avgc/=blocks;
      double total = k.ops_per_thread * threads * blocks;
      // ops per SM per cycle: 8 blocks per SM co-resident (256 thr x 8 = 2048)
      double per_sm_cycle = k.ops_per_thread * threads * 8 / avgc;
      printf("%-26s %8.3f ms  %10.3f Gop/s  %7.2f thread-ops/SM/cycle (clock64 basis)\n", k.name, ms, total/ms/1e6, per_sm_cycle);
    }
  }
  cudaError_t e = cudaGetLastError(); printf("status %s\n", cudaGetErrorString(e));
  return 0;
}
