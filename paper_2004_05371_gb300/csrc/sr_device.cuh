// Device-side building blocks of the hierarchical sum (sm_103a).
//
// Thread stage  : vector loads + per-lane register accumulation
//                 (summing(), Fig. "Basic function of device wide reduction").
// Warp stage    : __shfl_down_sync tree, offsets 16..1 (Section VII-D; the
//                 tile-shuffle form is the fastest correct warp reduction of
//                 Table V).
// Block stage   : warp leaders -> shared memory -> block barrier -> warp 0
//                 (block_reduce(), same figure; the final stage over at most
//                 32 values follows Table IV's "32 data points with a warp").
// Cluster stage : partials written into the rank-0 CTA's shared memory
//                 through distributed shared memory, then barrier.cluster.
// TMA bulk path : cp.async.bulk global->shared copies completing on mbarriers,
//                 every wait bounded by %globaltimer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cooperative_groups.h>

namespace sr {
namespace cg = cooperative_groups;

constexpr int kDtF32 = 0, kDtI32 = 1, kDtBF16 = 2, kDtFP8 = 3;
constexpr int kStageTwoKernel = 1, kStageAtomic = 2, kStageLastBlock = 3,
              kStageGridSync = 4, kStageSingle = 5;


// ------------------------------------------------------------------ loads
// Read-only streaming loads: no L1 allocation (each byte is used once).
__device__ __forceinline__ void ldg_vec(const void* p, uint32_t (&r)[4]) {
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "l"(p));
}
__device__ __forceinline__ void ldg_vec(const void* p, uint32_t (&r)[8]) {
    asm("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]),
          "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "l"(p));
}
__device__ __forceinline__ void lds_vec(uint32_t saddr, uint32_t (&r)[4]) {
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr));
}
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------ compensated pairs
// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no contraction:
// the explicit _rn intrinsics keep nvcc from fusing or reassociating).
struct Pair { float s, c; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// ------------------------------------------------------ value operations
// Accumulator / partial types: int64 (int32 input), float, Pair, double.
template <class A> struct Op;
template <> struct Op<long long> {
    __device__ static long long zero() { return 0; }
    __device__ static long long add(long long a, long long b) { return a + b; }
    __device__ static long long shfl_down(long long v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
    __device__ static long long shfl(long long v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    __device__ static long long shfl_up(long long v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
};
template <> struct Op<float> {
    __device__ static float zero() { return 0.f; }
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ static float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
    __device__ static float shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    __device__ static float shfl_up(float v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
};
template <> struct Op<double> {
    __device__ static double zero() { return 0.0; }
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
    __device__ static double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    __device__ static double shfl_up(double v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
};
template <> struct Op<Pair> {
    __device__ static Pair zero() { return Pair{0.f, 0.f}; }
    // (s1,c1) + (s2,c2): TwoSum of the leading parts, corrections added.
    __device__ static Pair add(Pair a, Pair b) {
        float s, e;
        two_sum(a.s, b.s, s, e);
        return Pair{s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
    }
    __device__ static Pair shfl_down(Pair v, int o) {
        return Pair{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
    }
    __device__ static Pair shfl(Pair v, int src) {
        return Pair{__shfl_sync(0xffffffffu, v.s, src), __shfl_sync(0xffffffffu, v.c, src)};
    }
    __device__ static Pair shfl_up(Pair v, int o) {
        return Pair{__shfl_up_sync(0xffffffffu, v.s, o), __shfl_up_sync(0xffffffffu, v.c, o)};
    }
};

template <class A> __device__ __forceinline__ A warp_reduce(A v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = Op<A>::add(v, Op<A>::shfl_down(v, o));
    return v;
}

// Block tree: the result is valid in thread 0.  `scratch` holds 32 values.
// Every thread of the block must call it (it contains block barriers).
template <class A> __device__ __forceinline__ A block_reduce(A v, A* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    v = warp_reduce(v);
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    A r = Op<A>::zero();
    if (warp == 0) {
        r = lane < nwarps ? scratch[lane] : Op<A>::zero();
        r = warp_reduce(r);
    }
    __syncthreads();
    return r;
}

// --------------------------------------------------------------- per-dtype
// Accumulator of the thread stage for each input type.
template <int DT, bool COMP> struct Acc { using T = float; };
template <> struct Acc<kDtI32, false> { using T = long long; };
template <int DT> struct Acc<DT, true> { using T = Pair; };

template <class A> __device__ __forceinline__ void acc_add_f(A& a, float v);
template <> __device__ __forceinline__ void acc_add_f<float>(float& a, float v) { a = __fadd_rn(a, v); }
template <> __device__ __forceinline__ void acc_add_f<Pair>(Pair& a, float v) {
    float s, e;
    two_sum(a.s, v, s, e);
    a.s = s;
    a.c = __fadd_rn(a.c, e);
}

// Add the elements packed in one 32-bit word into accumulator `a`.
template <int DT, class A> __device__ __forceinline__ void acc_word(A& a, uint32_t w);
template <> __device__ __forceinline__ void acc_word<kDtI32, long long>(long long& a, uint32_t w) {
    a += (long long)(int)w;
}
template <> __device__ __forceinline__ void acc_word<kDtF32, float>(float& a, uint32_t w) { acc_add_f(a, __uint_as_float(w)); }
template <> __device__ __forceinline__ void acc_word<kDtF32, Pair>(Pair& a, uint32_t w) { acc_add_f(a, __uint_as_float(w)); }
// BF16: each half of the word enters binary32 arithmetic through the
// mixed-precision add / sub (PTX `add.rn.f32.bf16`, sm_100+): d = a + c with a
// BF16 and c binary32, rounded once — the same result as widening a (exact:
// BF16 is the top 16 bits of a binary32) and adding, one instruction fewer.
// Measured: +4 % for the compensated form, unchanged plain.
__device__ __forceinline__ float bf16_lo_add(uint32_t w, float c) {
    float d;
    asm("{ .reg .b16 l, h; mov.b32 {l, h}, %1; add.rn.f32.bf16 %0, l, %2; }" : "=f"(d) : "r"(w), "f"(c));
    return d;
}
__device__ __forceinline__ float bf16_hi_add(uint32_t w, float c) {
    float d;
    asm("{ .reg .b16 l, h; mov.b32 {l, h}, %1; add.rn.f32.bf16 %0, h, %2; }" : "=f"(d) : "r"(w), "f"(c));
    return d;
}
__device__ __forceinline__ float bf16_lo_sub(uint32_t w, float c) {
    float d;
    asm("{ .reg .b16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.bf16 %0, l, %2; }" : "=f"(d) : "r"(w), "f"(c));
    return d;
}
__device__ __forceinline__ float bf16_hi_sub(uint32_t w, float c) {
    float d;
    asm("{ .reg .b16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.bf16 %0, h, %2; }" : "=f"(d) : "r"(w), "f"(c));
    return d;
}
template <> __device__ __forceinline__ void acc_word<kDtBF16, float>(float& a, uint32_t w) {
    a = bf16_hi_add(w, bf16_lo_add(w, a));  // low half first, as in memory order
}
// TwoSum(a.s, v) with v a BF16 half of w; both uses of v are mixed ops.
template <bool HI> __device__ __forceinline__ void acc_bf16_half(Pair& a, uint32_t w) {
    const float s = HI ? bf16_hi_add(w, a.s) : bf16_lo_add(w, a.s);
    const float bp = __fsub_rn(s, a.s);
    const float ap = __fsub_rn(s, bp);
    const float e = __fadd_rn(__fsub_rn(a.s, ap), HI ? bf16_hi_sub(w, bp) : bf16_lo_sub(w, bp));
    a.s = s;
    a.c = __fadd_rn(a.c, e);
}
template <> __device__ __forceinline__ void acc_word<kDtBF16, Pair>(Pair& a, uint32_t w) {
    acc_bf16_half<false>(a, w);
    acc_bf16_half<true>(a, w);
}
// FP8 E4M3: hardware conversion to f16x2 (exact: f16 covers the E4M3 range
// including its subnormals), then f16 -> f32 (exact).
template <class A> __device__ __forceinline__ void acc_word_fp8(A& a, uint32_t w) {
    __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
    __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&lo));
    float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&hi));
    acc_add_f(a, f0.x);
    acc_add_f(a, f0.y);
    acc_add_f(a, f1.x);
    acc_add_f(a, f1.y);
}
template <> __device__ __forceinline__ void acc_word<kDtFP8, float>(float& a, uint32_t w) {
    // the four values of a word sum exactly (see the compensated form below)
    __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
    __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&lo));
    float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&hi));
    a = __fadd_rn(a, __fadd_rn(__fadd_rn(f0.x, f0.y), __fadd_rn(f1.x, f1.y)));
}
// Compensated FP8: every E4M3 value is an integer multiple of 2^-9 below 2^9,
// so any sum of up to 64 of them is exact in binary32.  The four values of a
// word are therefore added plainly (exactly), and one TwoSum carries the
// word's total into the compensated accumulator.
template <> __device__ __forceinline__ void acc_word<kDtFP8, Pair>(Pair& a, uint32_t w) {
    __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
    __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&lo));
    float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&hi));
    acc_add_f(a, __fadd_rn(__fadd_rn(f0.x, f0.y), __fadd_rn(f1.x, f1.y)));
}

// One scalar element at index i of the input (head / tail of the vector body).
template <int DT, class A> __device__ __forceinline__ void acc_elem(A& a, const unsigned char* x, int64_t i);
template <> __device__ __forceinline__ void acc_elem<kDtI32, long long>(long long& a, const unsigned char* x, int64_t i) {
    a += (long long)reinterpret_cast<const int*>(x)[i];
}
template <class A> __device__ __forceinline__ void acc_elem_f32(A& a, const unsigned char* x, int64_t i) {
    acc_add_f(a, reinterpret_cast<const float*>(x)[i]);
}
template <class A> __device__ __forceinline__ void acc_elem_bf16(A& a, const unsigned char* x, int64_t i) {
    uint32_t b = reinterpret_cast<const unsigned short*>(x)[i];
    acc_add_f(a, __uint_as_float(b << 16));
}
template <class A> __device__ __forceinline__ void acc_elem_fp8(A& a, const unsigned char* x, int64_t i) {
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)x[i], __NV_E4M3);
    acc_add_f(a, __half2float(*reinterpret_cast<__half*>(&h)));
}
template <> __device__ __forceinline__ void acc_elem<kDtF32, float>(float& a, const unsigned char* x, int64_t i) { acc_elem_f32(a, x, i); }
template <> __device__ __forceinline__ void acc_elem<kDtF32, Pair>(Pair& a, const unsigned char* x, int64_t i) { acc_elem_f32(a, x, i); }
template <> __device__ __forceinline__ void acc_elem<kDtBF16, float>(float& a, const unsigned char* x, int64_t i) { acc_elem_bf16(a, x, i); }
template <> __device__ __forceinline__ void acc_elem<kDtBF16, Pair>(Pair& a, const unsigned char* x, int64_t i) { acc_elem_bf16(a, x, i); }
template <> __device__ __forceinline__ void acc_elem<kDtFP8, float>(float& a, const unsigned char* x, int64_t i) { acc_elem_fp8(a, x, i); }
template <> __device__ __forceinline__ void acc_elem<kDtFP8, Pair>(Pair& a, const unsigned char* x, int64_t i) { acc_elem_fp8(a, x, i); }

// ------------------------------------------------- thread-stage summation
// Add one loaded vector (W 32-bit words) into the W word accumulators.
template <int DT, class A, int W> struct AccVec {
    __device__ static __forceinline__ void run(A (&a)[W], const uint32_t (&v)[W]) {
#pragma unroll
        for (int w = 0; w < W; ++w) acc_word<DT>(a[w], v[w]);
    }
};
// Plain FP8: every E4M3 value is an integer multiple of 2^-9 of magnitude at
// most 448 (< 2^18 units of 2^-9), so up to 73 of them sum exactly in
// binary32.  A vector's 16 or 32 values are therefore summed exactly and
// added once, into word accumulator 0 (the others stay zero).
template <int W> struct AccVec<kDtFP8, float, W> {
    __device__ static __forceinline__ float word_sum(uint32_t w) {
        __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
        __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
        float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&lo));
        float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&hi));
        return __fadd_rn(__fadd_rn(f0.x, f0.y), __fadd_rn(f1.x, f1.y));
    }
    __device__ static __forceinline__ float vec_sum(const uint32_t (&v)[W]) {
        float t[W];
#pragma unroll
        for (int w = 0; w < W; ++w) t[w] = word_sum(v[w]);
#pragma unroll
        for (int s = W / 2; s >= 1; s >>= 1)
#pragma unroll
            for (int w = 0; w < s; ++w) t[w] = __fadd_rn(t[w], t[w + s]);
        return t[0];
    }
    __device__ static __forceinline__ void run(float (&a)[W], const uint32_t (&v)[W]) {
        a[0] = __fadd_rn(a[0], vec_sum(v));
    }
};

// Compensated FP8: the vector's values sum exactly (as above); one TwoSum
// carries the sum into the compensated accumulator 0.
template <int W> struct AccVec<kDtFP8, Pair, W> {
    __device__ static __forceinline__ void run(Pair (&a)[W], const uint32_t (&v)[W]) {
        acc_add_f(a[0], AccVec<kDtFP8, float, W>::vec_sum(v));
    }
};

// Two TwoSum accumulations at once in packed binary32 arithmetic (PTX
// add/sub.rn.f32x2, sm_100+): lane k computes s_k + v_k = t_k + e_k exactly
// (Knuth's TwoSum, each lane rounded to nearest like the scalar form) and
// adds e_k into c_k.  Half the issue slots of two scalar TwoSums.
__device__ __forceinline__ void two_sum2(float& s0, float& s1, float& c0, float& c1, float v0, float v1) {
    asm("{ .reg .b64 s, v, t, bp, ap, d1, d2, e, c;\n"
        " mov.b64 s, {%0, %1};\n mov.b64 c, {%2, %3};\n mov.b64 v, {%4, %5};\n"
        " add.rn.f32x2 t, s, v;\n sub.rn.f32x2 bp, t, s;\n sub.rn.f32x2 ap, t, bp;\n"
        " sub.rn.f32x2 d1, s, ap;\n sub.rn.f32x2 d2, v, bp;\n add.rn.f32x2 e, d1, d2;\n"
        " add.rn.f32x2 c, c, e;\n"
        " mov.b64 {%0, %1}, t;\n mov.b64 {%2, %3}, c; }"
        : "+f"(s0), "+f"(s1), "+f"(c0), "+f"(c1)
        : "f"(v0), "f"(v1));
}

// Compensated BF16: both halves of words w and w + 1 are widened exactly with
// integer operations (BF16 is the top half of a binary32) and accumulated two
// words at a time in packed arithmetic; each word accumulator still takes its
// low half, then its high half, so the result is that of the scalar form.
template <int W> struct AccVec<kDtBF16, Pair, W> {
    __device__ static __forceinline__ void run(Pair (&a)[W], const uint32_t (&v)[W]) {
#pragma unroll
        for (int w = 0; w < W; w += 2) {
            two_sum2(a[w].s, a[w + 1].s, a[w].c, a[w + 1].c, __uint_as_float(v[w] << 16),
                     __uint_as_float(v[w + 1] << 16));
            two_sum2(a[w].s, a[w + 1].s, a[w].c, a[w + 1].c, __uint_as_float(v[w] & 0xffff0000u),
                     __uint_as_float(v[w + 1] & 0xffff0000u));
        }
    }
};

// One batch of U loaded vectors into the accumulators: vector by vector,
// except FP8, whose values sum exactly in groups of up to 16 words (64
// values, below the 73 that always sum exactly): one addition per group.
template <int DT, class A, int W, int U> struct AccBatch {
    __device__ static __forceinline__ void run(A (&a)[W], const uint32_t (&v)[U][W]) {
#pragma unroll
        for (int u = 0; u < U; ++u) AccVec<DT, A, W>::run(a, v[u]);
    }
};
template <class A, int W, int U> struct AccBatch<kDtFP8, A, W, U> {
    static constexpr int kGroup = (16 / W) < U ? (16 / W) : U;  // vectors per exact group
    __device__ static __forceinline__ void run(A (&a)[W], const uint32_t (&v)[U][W]) {
#pragma unroll
        for (int g = 0; g < U; g += kGroup) {
            float t[kGroup];
#pragma unroll
            for (int k = 0; k < kGroup; ++k) t[k] = AccVec<kDtFP8, float, W>::vec_sum(v[g + k]);
#pragma unroll
            for (int s = kGroup / 2; s >= 1; s >>= 1)
#pragma unroll
                for (int k = 0; k < s; ++k) t[k] = __fadd_rn(t[k], t[k + s]);
            acc_add_f(a[0], t[0]);
        }
    }
};

// Dependent additions made into one word accumulator by one acc_word call.
template <int DT> struct AddsPerWord { static constexpr int v = 1; };   // F32, I32; FP8 (a vector sums exactly first)
template <> struct AddsPerWord<kDtBF16> { static constexpr int v = 2; };

// The thread stage keeps W word accumulators (one per 32-bit lane of its
// vector loads).  int64 sums are exact and compensated pairs carry their own
// error term: for them Levels does nothing and the words are folded in order
// at the end.  The plain binary32 form is blocked instead, so that no chain of
// dependent additions grows with n (a chain of k same-sign additions can err
// by ~k u |S|; on constant data 64 of them already exceed 4 eps32 |S|):
//   - a word accumulator takes at most kBlockAdds additions; then (flush) the
//     W words are folded pairwise into one block sum and restarted at zero;
//   - block sums enter level 1; every 16 blocks level 1 is added into level 2,
//     every 256 blocks level 2 into level 3.
// Every chain is then at most ~16 additions long up to 2^16 blocks per thread
// (2^20 values per word), and the thread's sum is ((fold + l1) + l2) + l3.
constexpr int kBlockAdds = 16;  // Levels<float> counts blocks in the upper bits of c, adds in the low 4

template <class A> struct Levels {
    __device__ __forceinline__ void init() {}
    template <int W> __device__ __forceinline__ void flush(A (&)[W]) {}
    template <int ADDS, int W> __device__ __forceinline__ void after(A (&)[W]) {}
    template <int W> __device__ __forceinline__ A total(const A (&a)[W]) const {
        A t = a[0];
#pragma unroll
        for (int w = 1; w < W; ++w) t = Op<A>::add(t, a[w]);
        return t;
    }
};

template <> struct Levels<float> {
    float l1, l2, l3;
    uint32_t c;  // (blocks << 4) | additions made into the words in this block
    __device__ __forceinline__ void init() {
        l1 = l2 = l3 = 0.f;
        c = 0u;
    }
    template <int W> __device__ __forceinline__ static float fold(float (&a)[W]) {
#pragma unroll
        for (int s = W / 2; s >= 1; s >>= 1)
#pragma unroll
            for (int w = 0; w < s; ++w) a[w] = __fadd_rn(a[w], a[w + s]);
        return a[0];
    }
    // Block sum into level 1 (block count already advanced in c), carries.
    template <int W> __device__ __forceinline__ void close(float (&a)[W]) {
        l1 = __fadd_rn(l1, fold(a));
#pragma unroll
        for (int w = 0; w < W; ++w) a[w] = 0.f;
        if ((c & 0xF0u) == 0u) {
            l2 = __fadd_rn(l2, l1);
            l1 = 0.f;
            if ((c & 0xFF0u) == 0u) {
                l3 = __fadd_rn(l3, l2);
                l2 = 0.f;
            }
        }
    }
    // End of a block whose length the caller controls.
    template <int W> __device__ __forceinline__ void flush(float (&a)[W]) {
        c = (c | 15u) + 1u;
        close(a);
    }
    // ADDS (a power of two <= kBlockAdds) additions were just made into each
    // word: the block closes when the low four bits of c carry, i.e. when
    // (c & 15) < ADDS after the addition.
    template <int ADDS, int W> __device__ __forceinline__ void after(float (&a)[W]) {
        static_assert(ADDS >= 1 && ADDS <= kBlockAdds && (ADDS & (ADDS - 1)) == 0, "block size");
        c += (uint32_t)ADDS;
        if ((c & 15u) < (uint32_t)ADDS) {
            c &= ~15u;
            close(a);
        }
    }
    template <int W> __device__ __forceinline__ float total(float (&a)[W]) const {
        return __fadd_rn(__fadd_rn(__fadd_rn(fold(a), l1), l2), l3);
    }
};

// ------------------------------------------------------------ partials
// A unit partial stored in the workspace: 16 bytes per slot.
//   int32 input          -> int64
//   float, no FP64 flag  -> float   (Pair when compensated)
//   FP64 combine         -> double  (s + c converted exactly term by term)
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(Pair v) { return (double)v.s + (double)v.c; }
__device__ __forceinline__ double to_double(long long v) { return (double)v; }
__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(Pair v) { return __fadd_rn(v.s, v.c); }

// ------------------------------------------- programmatic dependent launch
// A kernel launched with the programmatic-stream-serialisation attribute may
// start while the kernel before it in the stream is still running.
// grid_dependency_wait() blocks until that kernel has completed and its
// memory operations are visible (an immediate return for an ordinary launch),
// so it precedes every global-memory access; allow_dependents() lets the next
// such launch begin as soon as every CTA of this grid has issued it.  The
// kernel boundary stays a full barrier; only the launch latency overlaps.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ----------------------------------------------------------- mbarrier/TMA
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.  Returns
// false when `limit_ns` of %globaltimer time passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}
// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies (async proxy) into the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 1-D bulk copy global -> this CTA's shared memory; completes `bytes`
// transaction bytes on `bar`.  dst, src 16-byte aligned; bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

}  // namespace sr
