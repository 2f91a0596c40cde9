// Segmented (batched) sum: out[s] = sum of x[offsets[s] .. offsets[s+1]).
// Kernel templates, instantiated per input dtype by sr_segmented_<dtype>.cu.
//
// Work split: the concatenated range [offsets[0], offsets[nseg]) is cut into
// W equal, vector-aligned pieces of E elements, one per warp of the grid, so
// the load is balanced whatever the segment lengths.  Segment s is *owned*
// by the warp whose piece contains offsets[s].  Each warp
//   - sums the continuation of the segment that started before its piece
//     (its "first carry"),
//   - sums every segment it owns; a segment that ends inside the piece is
//     written to out directly, the one that runs past the end of the piece
//     leaves a "last carry".
// A segment spanning warps w_o..w_e is then finished as
//   out[s] = carry_last[w_o] + sum_{w = w_o+1..w_e} carry_first[w]
// in that fixed order (deterministic), after a grid-level join of one of four
// forms (the paper's Section VII-E barrier choice applied to the batch):
//   two-kernel  : a second kernel does every finish (implicit barrier);
//   grid.sync   : cooperative kernel, finishes after grid.sync();
//   last-block  : per-segment ticket; the last contributing warp finishes;
//   atomic      : spanning pieces atomically added into out (zeroed first).
#pragma once

#include <type_traits>

#include "sr_device.cuh"
#include "sr_kparams.h"

namespace sr {

template <int DT> struct SegElem { static constexpr int v = 4; };
template <> struct SegElem<kDtBF16> { static constexpr int v = 2; };
template <> struct SegElem<kDtFP8> { static constexpr int v = 1; };

// ------------------------------------------------------------ helpers
// First s in [0, nseg] with offsets[s] >= key (nseg if none).  Warp-wide:
// each round, 32 samples shrink the interval 32-fold.
__device__ __forceinline__ void lb_round(const int64_t* off, int64_t key, int lane, int64_t& lo, int64_t& hi) {
    if (hi - lo <= 32) return;
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t i = lo + (int64_t)lane * step;
    const bool pred = (i < hi) ? (__ldg(off + i) >= key) : true;
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (m == 0) {
        lo = lo + 31 * step + 1;
    } else {
        const int k = __ffs(m) - 1;
        const int64_t ik = lo + (int64_t)k * step;
        hi = ik < hi ? ik : hi;
        if (k > 0) lo = lo + (int64_t)(k - 1) * step + 1;
    }
}
// hi - lo <= 32 here.  With exactly 32 candidates left, every lane may hold
// an offset below the key: the ballot is then empty and the answer is hi.
__device__ __forceinline__ int64_t lb_final(const int64_t* off, int64_t key, int lane, int64_t lo, int64_t hi) {
    const int64_t i = lo + lane;
    const bool pred = (i < hi) ? (__ldg(off + i) >= key) : true;
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (m == 0) return hi;
    const int64_t r = lo + (__ffs(m) - 1);
    return r < hi ? r : hi;
}
__device__ __forceinline__ int64_t warp_lower_bound(const int64_t* off, int64_t nseg, int64_t key, int lane) {
    int64_t lo = 0, hi = nseg;  // answer in [lo, hi]
    while (hi - lo > 32) lb_round(off, key, lane, lo, hi);
    return lb_final(off, key, lane, lo, hi);
}

// Sum of x[a, b) by one warp; the result is valid in lane 0.
template <int DT, bool COMP, int VB, int UNROLL>
__device__ __forceinline__ typename Acc<DT, COMP>::T warp_piece_sum(const unsigned char* x, int64_t a, int64_t b,
                                                                    int lane) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int EB = SegElem<DT>::v;
    constexpr int PV = VB / EB;  // elements per vector
    constexpr int W = VB / 4;
    A acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = Op<A>::zero();
    if (b > a) {
        const uintptr_t addr = reinterpret_cast<uintptr_t>(x) + (uintptr_t)a * EB;
        const int64_t head = (int64_t)(((uintptr_t)VB - addr % VB) % VB) / EB;
        const int64_t va = a + (head < b - a ? head : b - a);
        const int64_t nv = (b - va) / PV;
        const int64_t tb = va + nv * PV;
        if (a + lane < va) acc_elem<DT>(acc[0], x, a + lane);
        const unsigned char* body = x + va * EB;
        int64_t v = lane;
        for (; v + (UNROLL - 1) * 32 < nv; v += UNROLL * 32) {
            uint32_t r[UNROLL][W];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) ldg_vec(body + (v + u * 32) * VB, r[u]);
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
#pragma unroll
                for (int w = 0; w < W; ++w) acc_word<DT>(acc[w], r[u][w]);
        }
        for (; v < nv; v += 32) {
            uint32_t r[W];
            ldg_vec(body + v * VB, r);
#pragma unroll
            for (int w = 0; w < W; ++w) acc_word<DT>(acc[w], r[w]);
        }
        if (tb + lane < b) acc_elem<DT>(acc[0], x, tb + lane);
    }
    A t = acc[0];
#pragma unroll
    for (int w = 1; w < W; ++w) t = Op<A>::add(t, acc[w]);
    return warp_reduce(t);
}

// ---------------------------------------------------- output and carries
__device__ __forceinline__ void seg_out(const SegParams& p, int64_t s, long long v) {
    reinterpret_cast<long long*>(p.out)[s] = v;
}
template <class A> __device__ __forceinline__ void seg_out(const SegParams& p, int64_t s, A v) {
    if (p.fp64) reinterpret_cast<double*>(p.out)[s] = __dmul_rn(to_double(v), (double)p.scale);
    else reinterpret_cast<float*>(p.out)[s] = __fmul_rn(to_float(v), p.scale);
}
__device__ __forceinline__ void seg_out_d(const SegParams& p, int64_t s, double v) {
    reinterpret_cast<double*>(p.out)[s] = __dmul_rn(v, (double)p.scale);
}
__device__ __forceinline__ void seg_atomic(const SegParams& p, int64_t s, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p.out) + s, (unsigned long long)v);
}
template <class A> __device__ __forceinline__ void seg_atomic(const SegParams& p, int64_t s, A v) {
    if (p.fp64) atomicAdd(reinterpret_cast<double*>(p.out) + s, __dmul_rn(to_double(v), (double)p.scale));
    else atomicAdd(reinterpret_cast<float*>(p.out) + s, __fmul_rn(to_float(v), p.scale));
}

template <class A> __device__ __forceinline__ void carry_store(const SegParams& p, unsigned char* arr, int64_t w, A v) {
    unsigned char* slot = arr + w * 16;
    if (p.fp64) *reinterpret_cast<double*>(slot) = to_double(v);
    else *reinterpret_cast<A*>(slot) = v;
}
template <> __device__ __forceinline__ void carry_store<long long>(const SegParams& p, unsigned char* arr, int64_t w,
                                                                   long long v) {
    (void)p;
    *reinterpret_cast<long long*>(arr + w * 16) = v;
}

template <class P> __device__ __forceinline__ P carry_load(const unsigned char* arr, int64_t w) {
    const unsigned char* s = arr + w * 16;
    if constexpr (std::is_same<P, Pair>::value) {
        float2 v = __ldcg(reinterpret_cast<const float2*>(s));
        return Pair{v.x, v.y};
    } else {
        return __ldcg(reinterpret_cast<const P*>(s));
    }
}

// Finish a spanning segment s owned by warp w_o, ending in warp w_e (whole
// warp calls; fixed order, so the result does not depend on which warp runs it).
template <class P> __device__ __forceinline__ void finish_span_typed(const SegParams& p, int64_t s, int64_t w_o,
                                                                     int64_t w_e, int lane) {
    P acc = Op<P>::zero();
    for (int64_t w = w_o + 1 + lane; w <= w_e; w += 32) acc = Op<P>::add(acc, carry_load<P>(p.carry_first, w));
    acc = warp_reduce(acc);
    if (lane == 0) {
        P total = Op<P>::add(carry_load<P>(p.carry_last, w_o), acc);
        if constexpr (std::is_same<P, double>::value) seg_out_d(p, s, total);
        else seg_out(p, s, total);
    }
}
template <class A> __device__ __forceinline__ void finish_span(const SegParams& p, int64_t s, int64_t w_o,
                                                               int64_t w_e, int lane) {
    if constexpr (std::is_same<A, long long>::value) {
        finish_span_typed<long long>(p, s, w_o, w_e, lane);
    } else {
        if (p.fp64) finish_span_typed<double>(p, s, w_o, w_e, lane);
        else finish_span_typed<A>(p, s, w_o, w_e, lane);
    }
}

// Per-segment ticket of the last-block form: every contributing warp
// arrives once; the last one finishes the segment and resets the ticket.
template <class A> __device__ __forceinline__ void span_arrive(const SegParams& p, int64_t s, int64_t w_o,
                                                               int64_t w_e, int lane) {
    unsigned t = 0;
    if (lane == 0) {
        __threadfence();
        t = atomicAdd(p.cnt + w_o, 1u);
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t == (unsigned)(w_e - w_o)) {
        __threadfence();
        finish_span<A>(p, s, w_o, w_e, lane);
        if (lane == 0) atomicExch(p.cnt + w_o, 0u);
    }
}

// ------------------------------------------------------------- main kernel
template <int DT, bool COMP, int VB, int UNROLL>
__global__ void __launch_bounds__(1024) seg_kernel(const SegParams p) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int PV = VB / SegElem<DT>::v;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t Wn = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t base = __ldg(p.offsets);
    const int64_t N = __ldg(p.offsets + p.nseg) - base;
    int64_t E = (N + Wn - 1) / Wn;
    E = ((E + PV - 1) / PV) * PV;
    if (E < PV) E = PV;
    const int64_t lo = base + (w * E < N ? w * E : N);
    const int64_t hi = base + ((w + 1) * E < N ? (w + 1) * E : N);

    // first segment starting at or after this piece; the owned segments are
    // those that start before the next piece (all remaining ones for the last warp)
    const int64_t s_begin = warp_lower_bound(p.offsets, p.nseg, base + w * E, lane);
    const int64_t next_lo = (w == Wn - 1) ? INT64_MAX : base + (w + 1) * E;

    // continuation of the segment that started before this piece
    if (lo < hi && s_begin > 0) {
        const int64_t cont_end = __ldg(p.offsets + s_begin);
        if (cont_end > lo) {
            const int64_t sp = s_begin - 1;
            const int64_t e = cont_end < hi ? cont_end : hi;
            A v = warp_piece_sum<DT, COMP, VB, UNROLL>(p.x, lo, e, lane);
            const int64_t w_o = (__ldg(p.offsets + sp) - base) / E;
            const int64_t w_e = (cont_end - 1 - base) / E;
            if (p.stage == kStageAtomic) {
                if (lane == 0) seg_atomic(p, sp, v);
            } else {
                if (lane == 0) carry_store(p, p.carry_first, w, v);
                if (p.stage == kStageLastBlock) span_arrive<A>(p, sp, w_o, w_e, lane);
            }
        }
    }

    // segments owned by this warp, offsets fetched 32 at a time
    int64_t spanning = -1;
    bool more = true;
    for (int64_t s0 = s_begin; more && s0 < p.nseg; s0 += 32) {
        const int64_t cnt = (p.nseg - s0) < 32 ? (p.nseg - s0) : 32;
        const int64_t my_end = (lane < cnt) ? __ldg(p.offsets + s0 + lane + 1) : 0;
        int64_t start = __ldg(p.offsets + s0);
        for (int k = 0; k < cnt; ++k) {
            if (start >= next_lo) {  // this segment belongs to the next piece
                more = false;
                break;
            }
            const int64_t end = __shfl_sync(0xffffffffu, my_end, k);
            const int64_t s = s0 + k;
            const int64_t e = end < hi ? end : hi;
            A v = warp_piece_sum<DT, COMP, VB, UNROLL>(p.x, start, e, lane);
            if (end <= hi) {
                if (lane == 0) seg_out(p, s, v);
            } else {  // runs past this piece: only the last owned segment can
                spanning = s;
                const int64_t w_e = (end - 1 - base) / E;
                if (p.stage == kStageAtomic) {
                    if (lane == 0) seg_atomic(p, s, v);
                } else {
                    if (lane == 0) carry_store(p, p.carry_last, w, v);
                    if (p.stage == kStageLastBlock) span_arrive<A>(p, s, w, w_e, lane);
                }
            }
            start = end;
        }
    }

    if (p.stage == kStageTwoKernel || p.stage == kStageGridSync) {
        if (lane == 0) p.last_seg[w] = spanning;
    }
    if (p.stage == kStageGridSync) {
        cg::grid_group g = cg::this_grid();
        if (!g.is_valid()) {
            if (threadIdx.x == 0) atomicOr(p.err, 2);
            return;
        }
        g.sync();
        if (spanning >= 0) {
            const int64_t end = __ldg(p.offsets + spanning + 1);
            finish_span<A>(p, spanning, w, (end - 1 - base) / E, lane);
        }
    }
}

// Second kernel of the two-kernel form: one warp per first-kernel warp.
template <int DT, bool COMP>
__global__ void __launch_bounds__(256) seg_finish_kernel(const SegParams p, int64_t Wn, int PV) {
    using A = typename Acc<DT, COMP>::T;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= Wn) return;
    const int64_t s = __ldcg(p.last_seg + w);
    if (s < 0) return;
    const int64_t base = __ldg(p.offsets);
    const int64_t N = __ldg(p.offsets + p.nseg) - base;
    int64_t E = (N + Wn - 1) / Wn;  // the first kernel's piece size
    E = ((E + PV - 1) / PV) * PV;
    if (E < PV) E = PV;
    const int64_t end = __ldg(p.offsets + s + 1);
    finish_span<A>(p, s, w, (end - 1 - base) / E, lane);
}

template <int DT, bool COMP, int VB>
inline const void* pick_seg(int unroll) {
    switch (unroll) {
    case 1: return (const void*)seg_kernel<DT, COMP, VB, 1>;
    case 2: return (const void*)seg_kernel<DT, COMP, VB, 2>;
    case 4: return (const void*)seg_kernel<DT, COMP, VB, 4>;
    case 8: return (const void*)seg_kernel<DT, COMP, VB, 8>;
    default: return nullptr;
    }
}

template <int DT, bool COMP>
inline bool pick_seg_kernels(int vec, int unroll, const void** main, const void** fin) {
    *main = vec == 16 ? pick_seg<DT, COMP, 16>(unroll) : (vec == 32 ? pick_seg<DT, COMP, 32>(unroll) : nullptr);
    *fin = (const void*)seg_finish_kernel<DT, COMP>;
    return *main != nullptr;
}

}  // namespace sr
