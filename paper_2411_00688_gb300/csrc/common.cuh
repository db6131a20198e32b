// Shared device helpers: dual-field storage types, Philox4x64-10, reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "kernels.hpp"

namespace tvs {

// ---------------------------------------------------------------- launches
// Every kernel is launched with programmatic dependent launch allowed (unless
// TVS_PDL=0): the next kernel in the stream may be scheduled while the previous
// one drains, and each kernel's first action, pdl_enter(), waits until the
// previous grid has completed and its memory is visible before touching any
// memory, then lets its own successor be scheduled.  The overlap hides the launch
// latency and ramp of the long chains of short, dependent kernels (thousands per
// solve); kernels not launched this way pass through pdl_enter() at no cost.
bool pdl_enabled();

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

template <typename... P, typename... A>
inline void launch_kernel(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  if (pdl_enabled()) {
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  // errors surface through cudaGetLastError() at the launcher's return
  (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// ---------------------------------------------------------------- storage
// The TV dual field may be stored as float, bfloat16, half or q15; arithmetic is
// always float32 and stores round to nearest (even).  ld/st move one value;
// ld2/st2 move two adjacent values (the first at an even element index, so the
// pair is aligned to its size); round / round2 give the value a store followed by
// a load would give, without the memory round trip; raw loads a stored value
// without decoding it, and cvt decodes one already held in a register.
//
// q15: signed 16-bit fixed point for values in [-1, 1], the range of every
// stored dual component (each is a component of a vector projected onto the unit
// ball).  The code i stands for i * fl(1/32767); a store clamps to [-1, 1] and
// takes i = the integer nearest (ties to even) to the exact product v * 32767.
// Both directions use only full-rate FP32 and integer instructions: with
// M = 1.5 * 2^23, the FFMA v * 32767 + M rounds to M + i exactly (|i| < 2^22),
// whose bit pattern is that of M plus i, and the float of i is the float with
// M's bits plus i, minus M.  Its absolute resolution, 2^-15 over the whole range,
// is 64 times finer than bfloat16's and 8 times finer than half's near |p| = 1,
// at the same two bytes.
struct q15 {
  int16_t v;
};
template <typename T> struct Elem;
template <> struct Elem<float> {
  static __device__ __forceinline__ float cvt(float v) { return v; }
  static __device__ __forceinline__ float raw(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ float ldc(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
  static __device__ __forceinline__ float round(float v) { return v; }
  static __device__ __forceinline__ float2 ld2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
  static __device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
  static __device__ __forceinline__ float2 round2(float2 v) { return v; }
};
template <> struct Elem<__nv_bfloat16> {
  static __device__ __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 raw(const __nv_bfloat16* p) { return __ldg(p); }
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ float ldc(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
  static __device__ __forceinline__ float2 ld2(const __nv_bfloat16* p) {
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
  }
  static __device__ __forceinline__ void st2(__nv_bfloat16* p, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v);
  }
  static __device__ __forceinline__ float2 round2(float2 v) { return __bfloat1622float2(__float22bfloat162_rn(v)); }
};
template <> struct Elem<__half> {
  static __device__ __forceinline__ float cvt(__half v) { return __half2float(v); }
  static __device__ __forceinline__ __half raw(const __half* p) { return __ldg(p); }
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ float ldc(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ float round(float v) { return __half2float(__float2half_rn(v)); }
  static __device__ __forceinline__ float2 ld2(const __half* p) {
    return __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
  }
  static __device__ __forceinline__ void st2(__half* p, float2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v); }
  static __device__ __forceinline__ float2 round2(float2 v) { return __half22float2(__float22half2_rn(v)); }
};
template <> struct Elem<q15> {
  static constexpr float kScale = 32767.f;
  static constexpr float kInv = 1.f / 32767.f;
  static constexpr float kMagic = 12582912.f;  // 1.5 * 2^23
  static constexpr int kMagicBits = 0x4B400000;
  static __device__ __forceinline__ float dec(int i) { return (__int_as_float(kMagicBits + i) - kMagic) * kInv; }
  static __device__ __forceinline__ int enc(float v) {
    return __float_as_int(__fmaf_rn(fminf(fmaxf(v, -1.f), 1.f), kScale, kMagic)) - kMagicBits;
  }
  static __device__ __forceinline__ float cvt(q15 v) { return dec(v.v); }
  static __device__ __forceinline__ q15 raw(const q15* p) { return q15{__ldg(reinterpret_cast<const short*>(p))}; }
  static __device__ __forceinline__ float ld(const q15* p) { return dec(__ldg(reinterpret_cast<const short*>(p))); }
  static __device__ __forceinline__ float ldc(const q15* p) { return dec(p->v); }
  static __device__ __forceinline__ void st(q15* p, float v) { p->v = (int16_t)enc(v); }
  // v is a projected component (|v| <= 1 up to float rounding, well inside the
  // half code step that the clamp of a store could change), so no clamp here
  static __device__ __forceinline__ float round(float v) { return (__fmaf_rn(v, kScale, kMagic) - kMagic) * kInv; }
  // sign extension of a 16-bit field by arithmetic alone: (f ^ 0x8000) - 0x8000
  static __device__ __forceinline__ int sx16(unsigned f) { return (int)(f ^ 0x8000u) - 0x8000; }
  static __device__ __forceinline__ float2 ld2(const q15* p) {
    const unsigned w = __ldg(reinterpret_cast<const unsigned*>(p));
    return make_float2(dec(sx16(w & 0xffffu)), dec(sx16(w >> 16)));
  }
  static __device__ __forceinline__ void st2(q15* p, float2 v) {
    *reinterpret_cast<unsigned*>(p) = ((unsigned)enc(v.x) & 0xffffu) | ((unsigned)enc(v.y) << 16);
  }
  static __device__ __forceinline__ float2 round2(float2 v) {
    const float2 m = make_float2(kMagic, kMagic);
    const float2 a = __fadd2_rn(__ffma2_rn(v, make_float2(kScale, kScale), m), make_float2(-kMagic, -kMagic));
    return __fmul2_rn(a, make_float2(kInv, kInv));
  }
};

// Calls f(TypeTag<T>{}) with T the storage type of dual dtype `dtype`.
template <typename T> struct TypeTag {
  using type = T;
};
template <typename F>
inline auto with_dual_type(int dtype, F&& f) {
  switch (dtype) {
    case DUAL_F32:
      return f(TypeTag<float>{});
    case DUAL_BF16:
      return f(TypeTag<__nv_bfloat16>{});
    case DUAL_F16:
      return f(TypeTag<__half>{});
    default:
      return f(TypeTag<q15>{});
  }
}

// ---------------------------------------------------------------- Philox4x64-10
// Counter-based generator of Salmon et al. (SC'11): per round,
// (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2, c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0),
// with the key bumped by the Weyl constants between rounds.
struct Philox4x64 {
  static constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull;
  static constexpr uint64_t M1 = 0xCA5A826395121157ull;
  static constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull;
  static constexpr uint64_t W1 = 0xBB67AE8584CAA73Bull;

  static __host__ __device__ inline void mulhilo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
#if defined(__CUDA_ARCH__)
    *lo = a * b;
    *hi = __umul64hi(a, b);
#else
    unsigned __int128 pr = (unsigned __int128)a * (unsigned __int128)b;
    *lo = (uint64_t)pr;
    *hi = (uint64_t)(pr >> 64);
#endif
  }

  static __host__ __device__ inline void block(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
      if (r > 0) { k0 += W0; k1 += W1; }
      uint64_t hi0, lo0, hi1, lo1;
      mulhilo(M0, c0, &hi0, &lo0);
      mulhilo(M1, c2, &hi1, &lo1);
      uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
      c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
  }

  // theta_k = [(w >> 11) < p 2^53], exact in double.
  static __host__ __device__ inline int coin(uint64_t seed, double p, uint64_t k) {
    uint64_t ctr[4] = {k, 0, 0, 0}, key[2] = {seed, 0}, out[4];
    block(ctr, key, out);
    return (double)(out[0] >> 11) < p * 9007199254740992.0 ? 1 : 0;
  }
};

// ---------------------------------------------------------------- reductions
// Compensated FP32 accumulator: s + c carries the running sum to about twice single
// precision (Knuth's TwoSum gives the exact rounding error of every addition, which
// c collects).  The objective and distance sums use it in place of FP64 arithmetic,
// whose throughput on this GPU is a small fraction of FP32's; its accuracy for
// sums of up to millions of FP32 terms is at the level of FP64 accumulation.  The
// intrinsics keep the compiler from fusing or reassociating the additions.
struct FAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ void add(float os, float oc) {
    add(os);
    c = __fadd_rn(c, oc);
  }
  __device__ __forceinline__ void add(const Partial& p) { add(p.s, p.c); }
};

template <int W>
__device__ __forceinline__ void warp_sum(FAcc& a) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    const float os = __shfl_down_sync(0xffffffffu, a.s, o);
    const float oc = __shfl_down_sync(0xffffffffu, a.c, o);
    a.add(os, oc);
  }
}

// Sums two per-thread accumulators over the block in a fixed order and writes the
// block totals to part_a[block_linear], part_b[block_linear] (deterministic).
template <int NT>
__device__ __forceinline__ void block_sum2_store(FAcc a, FAcc b, Partial* part_a, Partial* part_b,
                                                 int block_linear) {
  __shared__ Partial sa[NT / 32], sb[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum<32>(a);
  warp_sum<32>(b);
  if (lane == 0) {
    sa[warp] = Partial{a.s, a.c};
    sb[warp] = Partial{b.s, b.c};
  }
  __syncthreads();
  if (warp == 0) {
    a = FAcc();
    b = FAcc();
    if (lane < NT / 32) {
      a.s = sa[lane].s; a.c = sa[lane].c;
      b.s = sb[lane].s; b.c = sb[lane].c;
    }
    warp_sum<32>(a);
    warp_sum<32>(b);
    if (lane == 0) {
      if (part_a) part_a[block_linear] = Partial{a.s, a.c};
      if (part_b) part_b[block_linear] = Partial{b.s, b.c};
    }
  }
}

// Sum of n partials by one block of NT threads (fixed order); every thread gets
// the total as a double.
template <int NT>
__device__ __forceinline__ double block_sum_partials(const Partial* __restrict__ p, int n) {
  __shared__ Partial sp[NT / 32];
  __shared__ double total;
  FAcc a;
  for (int i = threadIdx.x; i < n; i += NT) a.add(p[i]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum<32>(a);
  if (lane == 0) sp[warp] = Partial{a.s, a.c};
  __syncthreads();
  if (warp == 0) {
    a = FAcc();
    if (lane < NT / 32) { a.s = sp[lane].s; a.c = sp[lane].c; }
    warp_sum<32>(a);
    if (lane == 0) total = (double)a.s + (double)a.c;
  }
  __syncthreads();
  return total;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Isotropic TV term of one pixel, |(D x)_i| = sqrt(dz^2 + dy^2 + dx^2), with one
// fixed rounding sequence so that every kernel produces identical per-pixel terms
// (dz = 0 for images: fma(0, 0, t) = t exactly).
__device__ __forceinline__ float tv_term(float dz, float dy, float dx) {
  return sqrtf(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
}

// Half-sample symmetric extension of index j into [0, n).
__device__ __forceinline__ int reflect_index(int j, int n) {
  if (j >= 0 && j < n) return j;
  const int period = 2 * n;
  j %= period;
  if (j < 0) j += period;
  return j >= n ? period - 1 - j : j;
}

}  // namespace tvs
