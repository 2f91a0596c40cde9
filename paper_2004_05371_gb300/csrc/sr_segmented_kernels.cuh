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
// The end of this file holds two forms without that split: whole segments
// per warp and whole segments per thread (no carries, no grid stage).
#pragma once

#include <type_traits>

#include "sr_device.cuh"
#include "sr_kparams.h"
#include "sr_segparams.h"

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

// Element j of a vector held as 32-bit words (the masked slow path; j is a
// compile-time constant after unrolling).
// Bits j of a PV-bit mask with a <= j < b (a and b clamped to [0, PV]).
template <int PV> __device__ __forceinline__ uint32_t run_mask(int64_t a, int64_t b) {
    const int ja = a <= 0 ? 0 : (a >= PV ? PV : (int)a);
    const int jb = b <= 0 ? 0 : (b >= PV ? PV : (int)b);
    const uint32_t below_b = jb >= 32 ? 0xffffffffu : (1u << jb) - 1u;
    const uint32_t below_a = ja >= 32 ? 0xffffffffu : (1u << ja) - 1u;
    return below_b & ~below_a;
}

// Sum of a lane's W word accumulators as a pairwise tree (log2 W dependent adds).
template <class A, int W> __device__ __forceinline__ A sum_words(const A (&acc)[W]) {
    A t[W];
#pragma unroll
    for (int k = 0; k < W; ++k) t[k] = acc[k];
#pragma unroll
    for (int h = 1; h < W; h <<= 1) {
#pragma unroll
        for (int k = 0; k + h < W; k += 2 * h) t[k] = Op<A>::add(t[k], t[k + h]);
    }
    return t[0];
}

template <int DT, class A> __device__ __forceinline__ void acc_vec_elem(A& a, const uint32_t* r, int j);
template <> __device__ __forceinline__ void acc_vec_elem<kDtI32, long long>(long long& a, const uint32_t* r, int j) {
    a += (long long)(int)r[j];
}
template <class A> __device__ __forceinline__ void acc_vec_elem_f32(A& a, const uint32_t* r, int j) {
    acc_add_f(a, __uint_as_float(r[j]));
}
template <class A> __device__ __forceinline__ void acc_vec_elem_bf16(A& a, const uint32_t* r, int j) {
    const uint32_t w = r[j >> 1];
    acc_add_f(a, __uint_as_float((j & 1) ? (w & 0xffff0000u) : (w << 16)));
}
template <class A> __device__ __forceinline__ void acc_vec_elem_fp8(A& a, const uint32_t* r, int j) {
    const uint32_t w = r[j >> 2];
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)((w >> (8 * (j & 3))) & 0xffu), __NV_E4M3);
    acc_add_f(a, __half2float(*reinterpret_cast<__half*>(&h)));
}
template <> __device__ __forceinline__ void acc_vec_elem<kDtF32, float>(float& a, const uint32_t* r, int j) { acc_vec_elem_f32(a, r, j); }
template <> __device__ __forceinline__ void acc_vec_elem<kDtF32, Pair>(Pair& a, const uint32_t* r, int j) { acc_vec_elem_f32(a, r, j); }
template <> __device__ __forceinline__ void acc_vec_elem<kDtBF16, float>(float& a, const uint32_t* r, int j) { acc_vec_elem_bf16(a, r, j); }
template <> __device__ __forceinline__ void acc_vec_elem<kDtBF16, Pair>(Pair& a, const uint32_t* r, int j) { acc_vec_elem_bf16(a, r, j); }
template <> __device__ __forceinline__ void acc_vec_elem<kDtFP8, float>(float& a, const uint32_t* r, int j) { acc_vec_elem_fp8(a, r, j); }
template <> __device__ __forceinline__ void acc_vec_elem<kDtFP8, Pair>(Pair& a, const uint32_t* r, int j) { acc_vec_elem_fp8(a, r, j); }

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
// One warp walks its piece [lo, hi) in element order: a scalar head up to the
// vector alignment, rows of 32 lane vectors (loads issued UNROLL rows ahead,
// independently of where segments end), and a scalar tail.  The current
// segment and its end travel with the walk; a row that contains no boundary
// is accumulated whole, a row that does takes a masked per-element path and
// emits each segment that ends in it — the load pipeline never drains at a
// boundary.
constexpr int kScanMin = 3;  // boundaries in a row from which the warp-wide pass pays

// BULK: the warp's vector body streams through its own ring of p.stages
// chunks of UNROLL rows in shared memory, one cp.async.bulk per chunk issued by
// lane 0 and completing on the chunk stage's mbarrier (every wait bounded by
// p.limit_ns; on expiry the warp records SR_ERR_TIMEOUT, waits for the copies
// it issued, and stops).  No registers hold rows in flight.
template <int DT, bool COMP, int VB, int UNROLL, bool DENSE, bool BULK>
__global__ void __launch_bounds__(512, 1) seg_kernel(const SegParams p) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int EB = SegElem<DT>::v;
    constexpr int PV = VB / EB;  // elements per lane vector
    constexpr int W = VB / 4;    // 32-bit words per lane vector
    constexpr int RW = 32 * PV;  // elements per row
    grid_dependency_wait();
    allow_dependents();
    if (p.bad != nullptr && __ldcg(p.bad) != 0) return;  // offsets failed the check: read nothing
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
    const int64_t next_lo = (w == Wn - 1) ? INT64_MAX : base + (w + 1) * E;

    // geometry of the piece: scalar head [lo, a0), vector rows [a0, hi_al), scalar tail [hi_al, hi)
    const uintptr_t addr = reinterpret_cast<uintptr_t>(p.x) + (uintptr_t)lo * EB;
    int64_t a0 = lo + (int64_t)(((uintptr_t)VB - addr % VB) % VB) / EB;
    if (a0 > hi) a0 = hi;
    const int64_t nvec = (hi - a0) / PV;
    const int64_t hi_al = a0 + nvec * PV;
    const int64_t nrows = (nvec + 31) / 32;
    const unsigned char* body = p.x + a0 * EB;

    // first batch of rows in flight before the segment search
    uint32_t buf[BULK ? 1 : UNROLL][W];
    constexpr uint32_t CHUNK = (uint32_t)UNROLL * 32u * VB;  // bytes of one ring stage
    const int64_t nchunks = (nrows + UNROLL - 1) / UNROLL;
    uint32_t ring = 0, bars = 0;
    // lane 0: copy chunk k of the body into its ring stage
    auto issue = [&](int64_t k) {
        const int64_t v0 = k * (UNROLL * 32);
        if (v0 >= nvec) return;
        const int64_t nv = (nvec - v0 < UNROLL * 32) ? nvec - v0 : (int64_t)UNROLL * 32;
        const int st = (int)(k % p.stages);
        mbar_arrive_expect_tx(bars + 8u * st, (uint32_t)(nv * VB));
        bulk_g2s(ring + (uint32_t)st * CHUNK, body + v0 * VB, (uint32_t)(nv * VB), bars + 8u * st);
    };
    if constexpr (BULK) {
        extern __shared__ __align__(128) unsigned char seg_dsm[];
        const int wib = threadIdx.x >> 5, nwib = blockDim.x >> 5;
        ring = smem_u32(seg_dsm) + (uint32_t)(wib * p.stages) * CHUNK;
        bars = smem_u32(seg_dsm) + (uint32_t)(nwib * p.stages) * CHUNK + (uint32_t)(wib * p.stages) * 8u;
        if (lane == 0) {
            for (int st = 0; st < p.stages; ++st) mbar_init(bars + 8u * st, 1);
            mbar_fence_init();
            for (int64_t k = 0; k < p.stages && k < nchunks; ++k) issue(k);
        }
        __syncwarp();
    } else {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t v = (int64_t)u * 32 + lane;
            if (v < nvec) ldg_vec(body + v * VB, buf[u]);
        }
    }

    const int64_t s_begin = warp_lower_bound(p.offsets, p.nseg, base + w * E, lane);
    // stream state (warp-uniform): segment `cur` = [cur_start, cur_end)
    int64_t cur = s_begin;
    if (lo < hi && s_begin > 0 && __ldg(p.offsets + s_begin) > lo) cur = s_begin - 1;  // continuation
    int64_t wb = cur + 1;  // offsets window: lane k holds offsets[wb + k]
    int64_t win = (wb + lane <= p.nseg) ? __ldg(p.offsets + wb + lane) : INT64_MAX;
    int64_t cur_start = (cur < p.nseg) ? __ldg(p.offsets + cur) : INT64_MAX;
    int64_t cur_end = (cur < p.nseg) ? __shfl_sync(0xffffffffu, win, 0) : INT64_MAX;
    int64_t spanning = -1;
    A acc[W];  // one accumulator per 32-bit word of the lane vector
#pragma unroll
    for (int k = 0; k < W; ++k) acc[k] = Op<A>::zero();

    // emit the current segment's piece and move to the next segment
    auto emit_advance = [&]() {
        A v = warp_reduce(sum_words<A, W>(acc));
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = Op<A>::zero();
        const int64_t s = cur;
        if (cur_start < lo) {  // continuation of a segment owned by an earlier warp
            if (p.stage == kStageAtomic) {
                if (lane == 0) seg_atomic(p, s, v);
            } else {
                if (lane == 0) carry_store(p, p.carry_first, w, v);
                if (p.stage == kStageLastBlock)
                    span_arrive<A>(p, s, (cur_start - base) / E, (cur_end - 1 - base) / E, lane);
            }
        } else if (cur_end <= hi) {  // owned and complete
            if (lane == 0) seg_out(p, s, v);
        } else {  // owned, runs past this piece
            spanning = s;
            if (p.stage == kStageAtomic) {
                if (lane == 0) seg_atomic(p, s, v);
            } else {
                if (lane == 0) carry_store(p, p.carry_last, w, v);
                if (p.stage == kStageLastBlock) span_arrive<A>(p, s, w, (cur_end - 1 - base) / E, lane);
            }
        }
        cur += 1;
        cur_start = cur_end;
        if (cur >= p.nseg) {
            cur_end = INT64_MAX;
            return;
        }
        if (cur + 1 - wb >= 32) {
            wb = cur + 1;
            win = (wb + lane <= p.nseg) ? __ldg(p.offsets + wb + lane) : INT64_MAX;
        }
        cur_end = __shfl_sync(0xffffffffu, win, (int)(cur + 1 - wb));
    };

    // A row [c0, c1) in which segments end, every boundary resolved in one
    // warp-wide pass: each lane splits its vector at the boundary it holds
    // (head before, tail from it on), a segmented inclusive scan over the lanes
    // (flag = the lane holds a boundary) yields the run open at the end of
    // every lane, and the lane holding boundary j emits the segment that ends
    // there: cur itself for j = 0 (with the rows before folded in; cur must be
    // owned by this warp, a continuation takes the per-segment path), an owned
    // segment complete inside the row for j >= 1.  The run open at the row's
    // end becomes the next segment's carry.  Applies when the row holds at
    // least kScanMin boundaries (below that one warp reduction per boundary is
    // cheaper than the pass's fixed ~17 shuffle rounds), no lane holds two,
    // and the offsets window already holds all of them; returns false, having
    // changed nothing, otherwise (no load is spent on a row that may fail).
    auto row_scan = [&](int64_t c0, int64_t c1, int64_t e0, bool valid, const uint32_t (&r_words)[W]) -> bool {
        if (cur_start < lo) return false;  // cur continues an earlier warp's segment: per-segment path
        const int kb = (int)(cur + 1 - wb);  // window lane of the row's first boundary
        const bool is_b = lane >= kb && win < c1;  // the row's boundaries: lanes kb .. kb + m - 1
        const unsigned bm = __ballot_sync(0xffffffffu, is_b);
        if (bm & 0x80000000u) return false;  // more boundaries may follow beyond the window
        const int m = __popc(bm);
        if (m < kScanMin) return false;
        const int tl = is_b ? (int)((win - c0) / PV) : -1;  // lane of the row holding boundary
        const int tl_next = __shfl_down_sync(0xffffffffu, tl, 1);
        if (__any_sync(0xffffffffu, is_b && lane < 31 && tl_next == tl)) return false;  // two in one lane
        const unsigned tmask = __reduce_or_sync(0xffffffffu, is_b ? (1u << tl) : 0u);
        const bool has_b = (tmask >> lane) & 1u;
        const int bj = __popc(tmask & ((1u << lane) - 1u));  // this lane's boundary among the row's
        const int64_t bpos = __shfl_sync(0xffffffffu, win, (kb + bj) & 31);
        const int q = has_b ? (int)(bpos - e0) : PV;  // elements j < q precede the boundary
        A head = Op<A>::zero(), tail = Op<A>::zero();
        if (valid) {
            const int jv = (c1 - e0 < PV) ? (int)(c1 - e0) : PV;  // elements of the lane inside the row
#pragma unroll
            for (int j = 0; j < PV; ++j) {
                if (j < jv) {
                    if (j < q) acc_vec_elem<DT>(head, r_words, j);
                    else acc_vec_elem<DT>(tail, r_words, j);
                }
            }
        }
        // segmented inclusive scan of the open runs over the lanes; before the
        // step with distance d a lane's partial covers lanes [lane - d + 1,
        // lane], which holds a boundary exactly when tmask has a bit there
        A x = has_b ? tail : head;
        const unsigned upto = (2u << lane) - 1u;  // lanes 0 .. lane (wraps to all ones at 31)
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const A xo = Op<A>::shfl_up(x, d);
            const int first = lane - d + 1 > 0 ? lane - d + 1 : 0;
            const bool f = (tmask & upto & ~((1u << first) - 1u)) != 0u;
            if (lane >= d && !f) x = Op<A>::add(xo, x);
        }
        A prev = Op<A>::shfl_up(x, 1);  // the run open at the end of the previous lane
        if (lane == 0) prev = Op<A>::zero();
        const A closed = Op<A>::add(prev, head);  // the segment ending at this lane's boundary
        const A open_end = Op<A>::shfl(x, 31);   // the run open at the row's end
        const int64_t last_pos = __shfl_sync(0xffffffffu, win, (kb + m - 1) & 31);
        const int64_t cur0 = cur;
        // owned segments complete inside the row (boundaries j >= 1)
        if (has_b && bj >= 1) seg_out(p, cur0 + bj, closed);
        // segment cur, owned by this warp and complete: the rows before this
        // one (acc, per lane) plus its part of this row
        const A first = Op<A>::shfl(closed, __ffs(tmask) - 1);
        A t = warp_reduce(sum_words<A, W>(acc));
        if (lane == 0) seg_out(p, cur0, Op<A>::add(t, first));
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = Op<A>::zero();
        // step over the segments emitted above to the one open at the row's end
        cur = cur0 + m;
        cur_start = last_pos;
        if (cur >= p.nseg) {
            cur_end = INT64_MAX;
        } else {
            const int64_t kc = cur + 1 - wb;
            if (kc < 32) {
                cur_end = __shfl_sync(0xffffffffu, win, (int)kc);
                if (kc >= 16) {  // refill the window ahead: the load overlaps the next rows
                    wb = cur + 1;
                    win = (wb + lane <= p.nseg) ? __ldg(p.offsets + wb + lane) : INT64_MAX;
                }
            } else {
                wb = cur + 1;
                win = (wb + lane <= p.nseg) ? __ldg(p.offsets + wb + lane) : INT64_MAX;
                cur_end = __shfl_sync(0xffffffffu, win, 0);
            }
        }
        if (lane == 0) acc[0] = open_end;
        return true;
    };

    // scalar chunk [c0, c1), at most 32 elements: lane l holds element c0 + l
    auto scalar_chunk = [&](int64_t c0, int64_t c1) {
        if (c0 >= c1) return;
        while (cur_end <= c0) emit_advance();
        const int64_t idx = c0 + lane;
        A one = Op<A>::zero();
        if (idx < c1) acc_elem<DT>(one, p.x, idx);
        for (;;) {
            if (idx < c1 && idx >= cur_start && idx < cur_end) acc[0] = Op<A>::add(acc[0], one);
            if (cur_end >= c1) break;
            emit_advance();
        }
    };

    // row r of vectors, words in `r_words` (lane's vector)
    auto row = [&](int64_t r, const uint32_t (&r_words)[W]) {
        const int64_t c0 = a0 + r * RW;
        const int64_t c1 = (c0 + RW < hi_al) ? c0 + RW : hi_al;
        while (cur_end <= c0) emit_advance();
        const int64_t e0 = c0 + (int64_t)lane * PV;
        const bool valid = e0 < c1;
        if (cur_end >= c1) {  // no boundary inside the row
            if (valid) {
#pragma unroll
                for (int k = 0; k < W; ++k) acc_word<DT>(acc[k], r_words[k]);
            }
            return;
        }
        if constexpr (DENSE) {
            if (row_scan(c0, c1, e0, valid, r_words)) return;
        }
        for (;;) {  // segments end inside this row (one reduction per segment)
            if (valid) {
                // element j of the lane's vector belongs to the current segment
                // when cur_start <= e0 + j < cur_end: one bit per j, from two
                // clamped offsets (static indices keep the vector in registers)
                const uint32_t m = run_mask<PV>(cur_start - e0, cur_end - e0);
#pragma unroll
                for (int j = 0; j < PV; ++j)
                    if ((m >> j) & 1u) acc_vec_elem<DT>(acc[j * W / PV], r_words, j);
            }
            if (cur_end >= c1) break;
            emit_advance();
        }
    };

    scalar_chunk(lo, a0);
    bool bail = false;
    if constexpr (BULK) {
        for (int64_t k = 0; k < nchunks; ++k) {
            const int st = (int)(k % p.stages);
            const uint32_t par = (uint32_t)((k / p.stages) & 1);
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(bars + 8u * st, par, p.limit_ns))) {
                if (lane == 0) {
                    atomicOr(p.err, kErrTimeout);
                    // leave no copy writing this CTA's shared memory: wait for the ones
                    // issued (chunks k .. k + stages - 1), bounded separately (>= 1 s)
                    const uint64_t drain = p.limit_ns > 1000000000ull ? p.limit_ns : 1000000000ull;
                    for (int64_t j = k; j < nchunks && j < k + p.stages; ++j)
                        mbar_wait_bounded(bars + 8u * (uint32_t)(j % p.stages), (uint32_t)((j / p.stages) & 1), drain);
                }
                bail = true;
                break;
            }
            const uint32_t sb = ring + (uint32_t)st * CHUNK + (uint32_t)lane * VB;
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int64_t r = k * UNROLL + u;
                if (r < nrows) {
                    uint32_t words[W];
#pragma unroll
                    for (int h = 0; h < W / 4; ++h) {
                        uint32_t t4[4];
                        lds_vec(sb + (uint32_t)u * 32u * VB + 16u * h, t4);
#pragma unroll
                        for (int i = 0; i < 4; ++i) words[4 * h + i] = t4[i];
                    }
                    row(r, words);
                }
            }
            __syncwarp();  // every lane has read the stage
            if (lane == 0) {
                fence_proxy_async_smem();
                issue(k + p.stages);
            }
        }
    } else {
        for (int64_t r = 0; r < nrows; r += UNROLL) {
            if (r > 0) {
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const int64_t v = (r + u) * 32 + lane;
                    if (v < nvec) ldg_vec(body + v * VB, buf[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
                if (r + u < nrows) row(r + u, buf[u]);
        }
    }
    if (!bail) {
        scalar_chunk(hi_al, hi);
        // the segment holding the piece's last element, then any (empty) segment
        // this warp owns that starts at or after hi
        while (cur < p.nseg && cur_start < next_lo) emit_advance();
    } else {
        spanning = -1;  // results are void (SR_ERR_TIMEOUT); nothing left to finish
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
    grid_dependency_wait();  // the implicit barrier: every first-kernel warp has finished
    allow_dependents();
    if (p.bad != nullptr && __ldcg(p.bad) != 0) return;
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

// The dense variant exists for at most 4 rows in flight per warp: with 8 its
// larger state through the hot loop cost 20-65 % on sparse layouts.
template <int DT, bool COMP, int VB, bool DENSE>
inline const void* pick_seg(int unroll) {
    switch (unroll) {
    case 1: return (const void*)seg_kernel<DT, COMP, VB, 1, DENSE, false>;
    case 2: return (const void*)seg_kernel<DT, COMP, VB, 2, DENSE, false>;
    case 4: return (const void*)seg_kernel<DT, COMP, VB, 4, DENSE, false>;
    case 8: return DENSE ? nullptr : (const void*)seg_kernel<DT, COMP, VB, 8, false, false>;
    default: return nullptr;
    }
}
// The TMA form: chunks of 2, 4 or 8 rows, no dense pass.
template <int DT, bool COMP, int VB>
inline const void* pick_seg_bulk(int unroll) {
    switch (unroll) {
    case 2: return (const void*)seg_kernel<DT, COMP, VB, 2, false, true>;
    case 4: return (const void*)seg_kernel<DT, COMP, VB, 4, false, true>;
    case 8: return (const void*)seg_kernel<DT, COMP, VB, 8, false, true>;
    default: return nullptr;
    }
}

template <int DT, bool COMP, bool DENSE>
inline const void* pick_seg_vec(int vec, int unroll) {
    return vec == 16 ? pick_seg<DT, COMP, 16, DENSE>(unroll)
                     : (vec == 32 ? pick_seg<DT, COMP, 32, DENSE>(unroll) : nullptr);
}

// The three kernel families of one dtype are instantiated in three
// translation units (sr_segmented_<dtype>{,_dense,_bulk}.cu) so they compile
// in parallel.
template <int DT, bool COMP>
inline const void* pick_seg_ldg(int vec, int unroll) { return pick_seg_vec<DT, COMP, false>(vec, unroll); }
template <int DT, bool COMP>
inline const void* pick_seg_dense(int vec, int unroll) { return pick_seg_vec<DT, COMP, true>(vec, unroll); }
template <int DT, bool COMP>
inline const void* pick_seg_tma(int vec, int unroll) {
    return vec == 16 ? pick_seg_bulk<DT, COMP, 16>(unroll) : (vec == 32 ? pick_seg_bulk<DT, COMP, 32>(unroll) : nullptr);
}

// ------------------------------------------------ lane-per-segment form
// Read-only 16-byte load that allocates in L1: for access patterns in which
// neighbouring lanes, or a lane's next load, use the rest of the line.
__device__ __forceinline__ void ldg_vec_l1(const void* p, uint32_t (&r)[4]) {
    asm("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(p));
}
__device__ __forceinline__ void ldg_vec_l1(const void* p, uint32_t (&r)[8]) {
    asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "l"(p));
}

// One thread sums x[s0, s1) alone: the VB-byte aligned body as VB-byte
// vectors (UNROLL per step, cached in L1: a lane's next vector and its
// neighbours' share the lines), the elements before and after it singly.
template <int DT, bool COMP, int VB, int UNROLL>
__device__ __forceinline__ typename Acc<DT, COMP>::T lane_sum(const unsigned char* x, int64_t s0, int64_t s1) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int EB = SegElem<DT>::v;
    constexpr int PV = VB / EB;  // elements per vector
    constexpr int W = VB / 4;    // 32-bit words per vector
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x);
    int64_t a0 = s0 + (int64_t)((((uintptr_t)VB - (xa + (uintptr_t)s0 * EB) % VB) % VB) / EB);
    if (a0 > s1) a0 = s1;
    const int64_t nv = (s1 - a0) / PV;
    const int64_t a1 = a0 + nv * PV;
    A edge = Op<A>::zero();  // head [s0, a0) and tail [a1, s1), fewer than PV each
    for (int64_t i = s0; i < a0; ++i) acc_elem<DT>(edge, x, i);
    for (int64_t i = a1; i < s1; ++i) acc_elem<DT>(edge, x, i);
    A acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = Op<A>::zero();
    const unsigned char* body = x + a0 * EB;
    int64_t v = 0;
    for (; v + UNROLL <= nv; v += UNROLL) {
        uint32_t r[UNROLL][W];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) ldg_vec_l1(body + (v + u) * VB, r[u]);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int q = 0; q < W; ++q) acc_word<DT>(acc[q], r[u][q]);
        }
    }
    for (; v < nv; ++v) {
        uint32_t r[W];
        ldg_vec_l1(body + v * VB, r);
#pragma unroll
        for (int q = 0; q < W; ++q) acc_word<DT>(acc[q], r[q]);
    }
    return Op<A>::add(sum_words<A, W>(acc), edge);
}

// SR_F_LANE_SEGMENTS: thread t of the grid sums segments t, t + T, ... alone
// (T threads), so a warp covers 32 consecutive segments: the offsets and the
// results move as coalesced words, and the lanes' loads fall into the warp's
// contiguous range.  One vector load replaces 16 / element-size scalar
// ones, which cut the time at 16-element segments 2.5-fold.  For very short
// segments only: a thread walks its segment alone.  No grid stage;
// deterministic.
template <int DT, bool COMP, int VB, int UNROLL>
__global__ void __launch_bounds__(512) seg_lane_kernel(const SegParams p) {
    grid_dependency_wait();
    allow_dependents();
    if (p.bad != nullptr && __ldcg(p.bad) != 0) return;  // offsets failed the check: read nothing
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < p.nseg; s += T) {
        const int64_t s0 = __ldg(p.offsets + s);
        const int64_t s1 = __ldg(p.offsets + s + 1);
        seg_out(p, s, lane_sum<DT, COMP, VB, UNROLL>(p.x, s0, s1));
    }
}

template <int DT, bool COMP, int VB>
inline const void* pick_seg_lane_u(int unroll) {
    switch (unroll) {
    case 1: return (const void*)seg_lane_kernel<DT, COMP, VB, 1>;
    case 2: return (const void*)seg_lane_kernel<DT, COMP, VB, 2>;
    case 4: return (const void*)seg_lane_kernel<DT, COMP, VB, 4>;
    case 8: return (const void*)seg_lane_kernel<DT, COMP, VB, 8>;
    default: return nullptr;
    }
}
template <int DT, bool COMP>
inline const void* pick_seg_lane(int vec, int unroll) {
    return vec == 16 ? pick_seg_lane_u<DT, COMP, 16>(unroll) : (vec == 32 ? pick_seg_lane_u<DT, COMP, 32>(unroll) : nullptr);
}

// ------------------------------------------------ warp-per-segment form
// SR_F_WARP_SEGMENTS: each warp sums whole segments, so no segment crosses a
// warp and there is no grid stage (results are deterministic).  Warps take
// blocks of G consecutive segments in turn (block b to warp b mod W, G =
// ceil(nseg / W) clamped to 1..32); lane k holds offsets[bG + k], so a block
// costs one coalesced offsets load.  Per segment, the elements before its
// first VB-aligned address and after its last whole vector are single loads
// by the first lanes; the vectors between are spread over the lanes, UNROLL
// per lane and batch; then one warp reduction and one store.  Segments go in
// pairs: both first batches are loaded before either is summed, so each warp
// keeps two segments' loads in flight.  A segment of at most kLaneAloneBytes
// is summed by its own lane instead (lane_sum), all such segments of a block
// at once: skewed layouts, mostly short segments with a long tail, pay the
// warp-wide path only for the long ones.
constexpr int64_t kLaneAloneBytes = 512;  // segments a lane of the warp form sums alone

// ------------------------------------------------------- adaptive form
// SR_F_ADAPTIVE_SEGMENTS: one cooperative launch for any layout.  Phase 1
// walks the segments in blocks as the warp form does and partitions them by
// length on the device: segments of at most kLaneAloneBytes go to single
// lanes, longer ones up to `thr` elements (kGroupMaxBytes, more for very
// large inputs) to groups of kGroupLanes lanes, and every longer segment is
// cut into chunks of `chunk` elements that are appended to a queue in the
// workspace.  grid.sync(), then phase 2: every warp takes
// chunks from the queue (one atomic per chunk) and sums them; the last chunk
// of a segment to finish combines the segment's chunk partials in chunk order,
// so the result does not depend on the order in which chunks were queued or
// taken (deterministic); a segment of one chunk is written directly.

// Queue the chunks of the block's long segments (whole warp calls).
__device__ __forceinline__ void enqueue_chunks(const SegParams& p, const SegQueue& q, int64_t b0, int64_t o,
                                               int64_t e, bool lng, int64_t chunk, int lane) {
    unsigned pend = __ballot_sync(0xffffffffu, lng);
    while (pend != 0u) {
        const int L = __ffs(pend) - 1;
        pend &= pend - 1u;
        const int64_t so = __shfl_sync(0xffffffffu, o, L);
        const int64_t se = __shfl_sync(0xffffffffu, e, L);
        const int64_t k = (se - so + chunk - 1) / chunk;
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(q.ctr, (unsigned)k);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((int64_t)base + k <= q.cap) {
            for (int64_t j = lane; j < k; j += 32) {
                q.desc[2 * ((int64_t)base + j)] = b0 + L;
                q.desc[2 * ((int64_t)base + j) + 1] = (j << 32) | k;
            }
            if (lane == 0) q.tick[base] = 0u;
        } else if (lane == 0) {
            atomicOr(p.err, kErrQueueFull);
        }
    }
}

// Adaptive form, mid-length segments: groups of kGroupLanes lanes, one
// segment per group, kGroupLanes / 32 segments per warp pass.  A load
// instruction of the warp then covers four 128-byte runs of four segments,
// and the fixed costs of a segment (offsets, head and tail, reduction) are
// shared by a quarter of the warp instead of all of it.
constexpr int kGroupLanes = 8;
constexpr int64_t kGroupMaxBytes = 8 << 10;  // longer ones: the whole warp, two at a time

// x[s0, s1) summed by the kGroupLanes lanes of a group (gl = lane in group):
// head and tail elements singly, the VB-aligned body strided over the group,
// UNROLL vectors per lane in flight.  Returns the lane's partial (reduce over
// the group afterwards, with the whole warp converged).
template <int DT, bool COMP, int VB, int UNROLL>
__device__ __forceinline__ typename Acc<DT, COMP>::T group_range_part(const unsigned char* x, int64_t s0,
                                                                       int64_t s1, int gl) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int EB = SegElem<DT>::v;
    constexpr int PV = VB / EB;
    constexpr int W = VB / 4;
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x);
    int64_t a0 = s0 + (int64_t)((((uintptr_t)VB - (xa + (uintptr_t)s0 * EB) % VB) % VB) / EB);
    if (a0 > s1) a0 = s1;
    const int64_t nv = (s1 - a0) / PV;
    const int64_t a1 = a0 + nv * PV;
    A edge = Op<A>::zero();
    for (int64_t i = s0 + gl; i < a0; i += kGroupLanes) acc_elem<DT>(edge, x, i);
    for (int64_t i = a1 + gl; i < s1; i += kGroupLanes) acc_elem<DT>(edge, x, i);
    A acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = Op<A>::zero();
    const unsigned char* body = x + a0 * EB;
    for (int64_t v0 = 0; v0 < nv; v0 += kGroupLanes * UNROLL) {
        uint32_t r[UNROLL][W];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t v = v0 + u * kGroupLanes + gl;
            if (v < nv) ldg_vec(body + v * VB, r[u]);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            if (v0 + u * kGroupLanes + gl < nv) AccVec<DT, A, W>::run(acc, r[u]);
    }
    return Op<A>::add(sum_words<A, W>(acc), edge);
}

// The block's mid-length segments (mask: lanes holding one), kGroupLanes
// lanes per segment, 32 / kGroupLanes at a time (whole warp calls).
template <int DT, bool COMP>
__device__ __forceinline__ void group_segments(const SegParams& p, int64_t b0, int64_t o, int64_t e, unsigned mask,
                                               int lane) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int NG = 32 / kGroupLanes;
    const int g = lane / kGroupLanes, gl = lane % kGroupLanes;
    while (mask != 0u) {
        // the next NG segments of the mask, one per group
        int mine = -1;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            const int L = mask ? __ffs(mask) - 1 : -1;
            if (L >= 0) mask &= mask - 1u;
            if (k == g) mine = L;
        }
        const int src = mine < 0 ? 0 : mine;
        const int64_t so = __shfl_sync(0xffffffffu, o, src);
        const int64_t se = __shfl_sync(0xffffffffu, e, src);
        A v = mine < 0 ? Op<A>::zero() : group_range_part<DT, COMP, 16, 4>(p.x, so, se, gl);
#pragma unroll
        for (int off = kGroupLanes / 2; off >= 1; off >>= 1) v = Op<A>::add(v, Op<A>::shfl_down(v, off));
        if (gl == 0 && mine >= 0) seg_out(p, b0 + mine, v);
    }
}

// One block of nb (<= 32) consecutive segments b0.. summed by one warp: lane
// k holds offsets[b0 + k], so the block costs one coalesced offsets load.
// Segments of at most kLaneAloneBytes are summed by their own lane; the rest
// by the whole warp, two at a time.  ADAPT (the adaptive form): segments
// longer than `thr` elements are queued as chunks of `chunk` elements, the
// others beyond kLaneAloneBytes go to lane groups (no whole-warp path).
template <int DT, bool COMP, int VB, int UNROLL, bool ADAPT>
__device__ __forceinline__ void seg_warp_block(const SegParams& p, const SegQueue* q, int64_t b0, int64_t nb,
                                               int lane, int64_t thr, int64_t chunk) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int EB = SegElem<DT>::v;
    constexpr int PV = VB / EB;  // elements per lane vector
    constexpr int W = VB / 4;    // 32-bit words per lane vector
    const uintptr_t xa = reinterpret_cast<uintptr_t>(p.x);
    const int64_t i = b0 + (lane < nb ? lane : nb);           // lane nb (or 31) holds the end
    const int64_t o = __ldg(p.offsets + i);
    const int64_t o_end = __ldg(p.offsets + b0 + nb);
    // this lane's segment [o, e); the short ones are summed by their lane alone
    const int64_t o_up = __shfl_down_sync(0xffffffffu, o, 1);
    const bool mine = lane < nb;
    const int64_t e = (lane + 1 < nb) ? o_up : o_end;
    const bool alone = mine && (e - o) * EB <= kLaneAloneBytes;
    if (alone) seg_out(p, b0 + lane, lane_sum<DT, COMP, 16, 4>(p.x, o, e));
    if constexpr (ADAPT) {
        // adaptive form: segments longer than `thr` elements go to the chunk
        // queue, the others to lane groups
        const bool lng = mine && (e - o) > thr;
        enqueue_chunks(p, *q, b0, o, e, lng, chunk, lane);
        group_segments<DT, COMP>(p, b0, o, e, __ballot_sync(0xffffffffu, mine && !alone && !lng), lane);
        return;
    }
    // the rest by the whole warp, two at a time: both first batches of loads in flight together
    unsigned todo = __ballot_sync(0xffffffffu, mine && !alone);
    while (todo != 0u) {
        const int k0 = __ffs(todo) - 1;
        todo &= todo - 1u;
        const bool two = todo != 0u;  // warp-uniform
        const int k1 = two ? __ffs(todo) - 1 : k0;
        if (two) todo &= todo - 1u;
        int64_t s0[2], s1[2];
        s0[0] = __shfl_sync(0xffffffffu, o, k0);
        s1[0] = __shfl_sync(0xffffffffu, e, k0);
        s0[1] = __shfl_sync(0xffffffffu, o, k1);
        s1[1] = __shfl_sync(0xffffffffu, e, k1);
        if (!two) s0[1] = s1[1] = s1[0];  // an empty second segment
        int64_t a0[2], nv[2];
        A edge[2], acc[2][W];
        uint32_t r[2][UNROLL][W];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            a0[j] = s0[j] + (int64_t)((((uintptr_t)VB - (xa + (uintptr_t)s0[j] * EB) % VB) % VB) / EB);
            if (a0[j] > s1[j]) a0[j] = s1[j];
            nv[j] = (s1[j] - a0[j]) / PV;
            const int64_t a1 = a0[j] + nv[j] * PV;
            edge[j] = Op<A>::zero();  // head [s0, a0) and tail [a1, s1), fewer than PV each
            if (lane < a0[j] - s0[j]) acc_elem<DT>(edge[j], p.x, s0[j] + lane);
            if (lane < s1[j] - a1) acc_elem<DT>(edge[j], p.x, a1 + lane);
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int64_t v = u * 32 + lane;
                if (v < nv[j]) ldg_vec(p.x + (a0[j] + v * PV) * EB, r[j][u]);
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int q = 0; q < W; ++q) acc[j][q] = Op<A>::zero();
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if (u * 32 + lane < nv[j]) {
#pragma unroll
                    for (int q = 0; q < W; ++q) acc_word<DT>(acc[j][q], r[j][u][q]);
                }
            }
        }
        // the rest of a segment longer than one batch, with both batch
        // buffers free now: 2 * UNROLL vectors per lane in flight
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const unsigned char* body = p.x + a0[j] * EB;
            for (int64_t v0 = 32 * UNROLL; v0 < nv[j]; v0 += 64 * UNROLL) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int u = 0; u < UNROLL; ++u) {
                        const int64_t v = v0 + (h * UNROLL + u) * 32 + lane;
                        if (v < nv[j]) ldg_vec(body + v * VB, r[h][u]);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int u = 0; u < UNROLL; ++u) {
                        if (v0 + (h * UNROLL + u) * 32 + lane < nv[j]) {
#pragma unroll
                            for (int q = 0; q < W; ++q) acc_word<DT>(acc[j][q], r[h][u][q]);
                        }
                    }
                }
            }
        }
        const A t0 = warp_reduce(Op<A>::add(sum_words<A, W>(acc[0]), edge[0]));
        const A t1 = warp_reduce(Op<A>::add(sum_words<A, W>(acc[1]), edge[1]));
        if (lane == 0) {
            seg_out(p, b0 + k0, t0);
            if (two) seg_out(p, b0 + k1, t1);
        }
    }
}

template <int DT, bool COMP, int VB, int UNROLL>
__global__ void __launch_bounds__(512) seg_warp_kernel(const SegParams p) {
    grid_dependency_wait();
    allow_dependents();
    if (p.bad != nullptr && __ldcg(p.bad) != 0) return;  // offsets failed the check: read nothing
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t Wn = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t G = (p.nseg + Wn - 1) / Wn;
    G = G < 1 ? 1 : (G > 32 ? 32 : G);
    for (int64_t b0 = w * G; b0 < p.nseg; b0 += Wn * G)
        seg_warp_block<DT, COMP, VB, UNROLL, false>(p, nullptr, b0, (p.nseg - b0 < G) ? p.nseg - b0 : G, lane, 0, 0);
}

// x[s0, s1) summed by one warp: the elements before the first VB-aligned
// address and after the last whole vector singly by the first lanes, the
// vectors between strided over the lanes, UNROLL per lane in flight; blocked
// accumulation (Levels) in the plain binary32 form; warp reduction.
template <int DT, bool COMP, int VB, int UNROLL>
__device__ __forceinline__ typename Acc<DT, COMP>::T warp_range_sum(const unsigned char* x, int64_t s0, int64_t s1,
                                                                     int lane) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int EB = SegElem<DT>::v;
    constexpr int PV = VB / EB;
    constexpr int W = VB / 4;
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x);
    int64_t a0 = s0 + (int64_t)((((uintptr_t)VB - (xa + (uintptr_t)s0 * EB) % VB) % VB) / EB);
    if (a0 > s1) a0 = s1;
    const int64_t nv = (s1 - a0) / PV;
    const int64_t a1 = a0 + nv * PV;
    A edge = Op<A>::zero();
    if (lane < a0 - s0) acc_elem<DT>(edge, x, s0 + lane);
    if (lane < s1 - a1) acc_elem<DT>(edge, x, a1 + lane);
    A acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = Op<A>::zero();
    Levels<A> lv;
    lv.init();
    const unsigned char* body = x + a0 * EB;
    for (int64_t v0 = 0; v0 < nv; v0 += 32 * UNROLL) {
        uint32_t r[UNROLL][W];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t v = v0 + u * 32 + lane;
            if (v < nv) ldg_vec(body + v * VB, r[u]);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            if (v0 + u * 32 + lane < nv) AccVec<DT, A, W>::run(acc, r[u]);
        lv.template after<UNROLL * AddsPerWord<DT>::v>(acc);
    }
    return warp_reduce(Op<A>::add(lv.total(acc), edge));
}

// The last chunk of segment s to finish: partials [base, base + k) in
// chunk order (lane-strided, then the warp tree), written to out[s].
template <class P> __device__ __forceinline__ void combine_chunks_typed(const SegParams& p, const SegQueue& q,
                                                                        int64_t s, int64_t base, int64_t k, int lane) {
    P acc = Op<P>::zero();
    for (int64_t j = lane; j < k; j += 32) acc = Op<P>::add(acc, carry_load<P>(q.part, base + j));
    acc = warp_reduce(acc);
    if (lane == 0) {
        if constexpr (std::is_same<P, double>::value) seg_out_d(p, s, acc);
        else seg_out(p, s, acc);
    }
}
template <class A> __device__ __forceinline__ void combine_chunks(const SegParams& p, const SegQueue& q, int64_t s,
                                                                  int64_t base, int64_t k, int lane) {
    if constexpr (std::is_same<A, long long>::value) {
        combine_chunks_typed<long long>(p, q, s, base, k, lane);
    } else {
        if (p.fp64) combine_chunks_typed<double>(p, q, s, base, k, lane);
        else combine_chunks_typed<A>(p, q, s, base, k, lane);
    }
}

constexpr int kAdaptStreamVB = 32, kAdaptStreamUnroll = 4;  // phase 2: 4 KiB per warp in flight

// Launched cooperatively with at most the resident number of CTAs.  VB and
// UNROLL shape phase 1's whole-warp segments (as the warp form).
template <int DT, bool COMP, int VB, int UNROLL>
__global__ void __launch_bounds__(256, 4) seg_adaptive_kernel(const SegParams p, const SegQueue q) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int EB = SegElem<DT>::v;
    grid_dependency_wait();
    allow_dependents();
    if (p.bad != nullptr && __ldcg(p.bad) != 0) return;  // every thread, before any grid barrier
    cg::grid_group g = cg::this_grid();
    if (!g.is_valid()) {  // not launched cooperatively: never wait
        if (threadIdx.x == 0) atomicOr(p.err, kErrNotCooperative);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t Wn = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // queue threshold and chunk size (elements): a queued segment of length L
    // takes at most L / chunk + 1 <= L / chunk + L / thr chunks, so with both
    // at least 2 total / capacity the queue cannot overflow
    const int64_t total = __ldg(p.offsets + p.nseg) - __ldg(p.offsets);
    const int64_t need = (2 * total + q.cap - 1) / q.cap;
    int64_t thr = kGroupMaxBytes / EB;
    if (thr < need) thr = need;
    int64_t chunk = kAdaptChunkBytes / EB;
    if (chunk < thr) chunk = thr;
    chunk = (chunk + 31) / 32 * 32;

    // phase 1: blocks of G consecutive segments, block b to warp b mod Wn
    int64_t G = (p.nseg + Wn - 1) / Wn;
    G = G < 1 ? 1 : (G > 32 ? 32 : G);
    for (int64_t b0 = w * G; b0 < p.nseg; b0 += Wn * G)
        seg_warp_block<DT, COMP, VB, UNROLL, true>(p, &q, b0, (p.nseg - b0 < G) ? p.nseg - b0 : G, lane, thr, chunk);

    g.sync();  // every long segment's chunks are queued

    // phase 2: chunks from the queue
    const int64_t nq = min((int64_t)__ldcg(q.ctr), q.cap);
    unsigned idx = 0;
    if (lane == 0) idx = atomicAdd(q.ctr + 1, 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    // the current chunk's descriptor and offsets are read one chunk ahead:
    // lane 0 holds (segment, j | k, segment start, end) of the next chunk
    int64_t ds = 0, de = 0;
    long long djk = 0, dsg = 0;
    if (lane == 0 && (int64_t)idx < nq) {
        dsg = __ldcg(q.desc + 2 * (int64_t)idx);
        djk = __ldcg(q.desc + 2 * (int64_t)idx + 1);
        ds = __ldg(p.offsets + dsg);
        de = __ldg(p.offsets + dsg + 1);
    }
    while ((int64_t)idx < nq) {
        const int64_t s = __shfl_sync(0xffffffffu, dsg, 0);
        const long long jk = __shfl_sync(0xffffffffu, djk, 0);
        const int64_t o = __shfl_sync(0xffffffffu, ds, 0), e = __shfl_sync(0xffffffffu, de, 0);
        const int64_t j = jk >> 32, k = jk & 0xffffffffll;
        unsigned nxt = 0;
        if (lane == 0) {  // the next chunk and its descriptor, while this one is summed
            nxt = atomicAdd(q.ctr + 1, 1u);
            if ((int64_t)nxt < nq) {
                dsg = __ldcg(q.desc + 2 * (int64_t)nxt);
                djk = __ldcg(q.desc + 2 * (int64_t)nxt + 1);
                ds = __ldg(p.offsets + dsg);
                de = __ldg(p.offsets + dsg + 1);
            }
        }
        const int64_t c0 = o + j * chunk;
        const int64_t c1 = c0 + chunk < e ? c0 + chunk : e;
        const A v = warp_range_sum<DT, COMP, kAdaptStreamVB, kAdaptStreamUnroll>(p.x, c0, c1, lane);
        const int64_t base = (int64_t)idx - j;
        if (k == 1) {  // a segment of one chunk: no partial, no ticket
            if (lane == 0) seg_out(p, s, v);
            idx = __shfl_sync(0xffffffffu, nxt, 0);
            continue;
        }
        unsigned t = 0;
        if (lane == 0) {
            carry_store(p, q.part, (int64_t)idx, v);
            __threadfence();
            t = atomicAdd(q.tick + base, 1u);
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((int64_t)t == k - 1) {  // the segment's last chunk: combine in chunk order
            __threadfence();
            combine_chunks<A>(p, q, s, base, k, lane);
        }
        idx = __shfl_sync(0xffffffffu, nxt, 0);
    }
    // the last warp out resets the counters for the next launch
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(q.ctr + 2, 1u) == (unsigned)(Wn - 1)) {
            q.ctr[0] = 0u;
            q.ctr[1] = 0u;
            q.ctr[2] = 0u;
            __threadfence();
        }
    }
}

// Phase 1 runs the warp form's default shape (16-byte vectors, 2 per lane).
template <int DT, bool COMP>
inline const void* pick_seg_adapt(int vec, int unroll) {
    return (vec == 16 && unroll == 2) ? (const void*)seg_adaptive_kernel<DT, COMP, 16, 2> : nullptr;
}

template <int DT, bool COMP, int VB>
inline const void* pick_seg_warp_u(int unroll) {
    switch (unroll) {
    case 1: return (const void*)seg_warp_kernel<DT, COMP, VB, 1>;
    case 2: return (const void*)seg_warp_kernel<DT, COMP, VB, 2>;
    case 4: return (const void*)seg_warp_kernel<DT, COMP, VB, 4>;
    case 8: return (const void*)seg_warp_kernel<DT, COMP, VB, 8>;
    default: return nullptr;
    }
}
template <int DT, bool COMP>
inline const void* pick_seg_warp(int vec, int unroll) {
    return vec == 16 ? pick_seg_warp_u<DT, COMP, 16>(unroll) : (vec == 32 ? pick_seg_warp_u<DT, COMP, 32>(unroll) : nullptr);
}

}  // namespace sr
