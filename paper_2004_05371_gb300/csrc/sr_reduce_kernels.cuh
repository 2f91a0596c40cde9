// Single-array hierarchical sum: kernel templates.  Included once per input
// dtype by sr_reduce_<dtype>.cu, which instantiates them.
//
// Stages of one launch (paper Section VII-E, Figs. "Basic function of device
// wide reduction", "... explicit device synchronization", "... implicit
// device synchronization"):
//   1. thread : grid-stride vector loads (LDG path) or a TMA bulk-copy ring in
//               shared memory (BULK path), accumulated per 32-bit lane;
//   2. warp   : shuffle tree;
//   3. block  : shared memory + __syncthreads, warp 0 finishes;
//   4. cluster: DSMEM writes into rank 0, barrier.cluster, rank 0 finishes;
//   5. grid   : two-kernel | atomic | last-block-done | grid.sync | none.
#pragma once

#include <type_traits>

#include "sr_device.cuh"
#include "sr_kparams.h"

namespace sr {

template <int DT> struct ElemBytes { static constexpr int v = 4; };
template <> struct ElemBytes<kDtBF16> { static constexpr int v = 2; };
template <> struct ElemBytes<kDtFP8> { static constexpr int v = 1; };

// ------------------------------------------------------- partial storage
template <class P> __device__ __forceinline__ void slot_store(unsigned char* slot, P v) {
    *reinterpret_cast<P*>(slot) = v;
}
template <class P> __device__ __forceinline__ P slot_load(const unsigned char* slot);
template <> __device__ __forceinline__ long long slot_load<long long>(const unsigned char* s) {
    return __ldcg(reinterpret_cast<const long long*>(s));
}
template <> __device__ __forceinline__ float slot_load<float>(const unsigned char* s) {
    return __ldcg(reinterpret_cast<const float*>(s));
}
template <> __device__ __forceinline__ double slot_load<double>(const unsigned char* s) {
    return __ldcg(reinterpret_cast<const double*>(s));
}
template <> __device__ __forceinline__ Pair slot_load<Pair>(const unsigned char* s) {
    float2 v = __ldcg(reinterpret_cast<const float2*>(s));
    return Pair{v.x, v.y};
}

// ------------------------------------------------------------ the output
__device__ __forceinline__ void out_write(long long v, const KParams& p) { *reinterpret_cast<long long*>(p.out) = v; }
__device__ __forceinline__ void out_write(float v, const KParams& p) {
    *reinterpret_cast<float*>(p.out) = __fmul_rn(v, p.scale);
}
__device__ __forceinline__ void out_write(Pair v, const KParams& p) { out_write(to_float(v), p); }
__device__ __forceinline__ void out_write(double v, const KParams& p) {
    *reinterpret_cast<double*>(p.out) = __dmul_rn(v, (double)p.scale);
}

__device__ __forceinline__ void out_atomic(long long v, const KParams& p) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p.out), (unsigned long long)v);
}
template <class A> __device__ __forceinline__ void out_atomic(A v, const KParams& p) {
    if (p.fp64)
        atomicAdd(reinterpret_cast<double*>(p.out), __dmul_rn(to_double(v), (double)p.scale));
    else
        atomicAdd(reinterpret_cast<float*>(p.out), __fmul_rn(to_float(v), p.scale));
}

// Reduce the unit partial slots in a fixed order (deterministic, whichever
// unit runs it) and write the result.  Whole block participates.
template <class P> __device__ __forceinline__ void reduce_slots(const KParams& p) {
    __shared__ __align__(16) unsigned char scratch_raw[32 * sizeof(P)];
    // blocks of kBlockAdds slots per thread (binary32: no long same-sign chain)
    P acc[1] = {Op<P>::zero()};
    Levels<P> lv;
    lv.init();
    int n = 0;
    for (int i = threadIdx.x; i < p.units; i += blockDim.x) {
        acc[0] = Op<P>::add(acc[0], slot_load<P>(p.partials + (size_t)i * 16));
        if (++n == kBlockAdds) {
            lv.flush(acc);
            n = 0;
        }
    }
    P v = block_reduce(lv.total(acc), reinterpret_cast<P*>(scratch_raw));
    if (threadIdx.x == 0) out_write(v, p);
}

// Compensated unit partials: the (sum, correction) pairs are combined in
// binary32 pair arithmetic, whose error is at most about units * u^2 *
// sum|s_i| (u = 2^-24: each pair addition rounds only its correction terms).
// With fp64_auto set, when that bound could exceed 1e-6 |S| the block
// recombines the partials in binary64 (fixed order) before writing the
// binary32 result — binary64 only in the cross-unit combine, only when the
// compensated bound is not met.
template <> __device__ __forceinline__ void reduce_slots<Pair>(const KParams& p) {
    __shared__ __align__(16) unsigned char scratch_raw[32 * sizeof(double)];
    __shared__ int s_redo;
    Pair v = Op<Pair>::zero();
    float a = 0.f;
    for (int i = threadIdx.x; i < p.units; i += blockDim.x) {
        const Pair q = slot_load<Pair>(p.partials + (size_t)i * 16);
        v = Op<Pair>::add(v, q);
        a = __fadd_rn(a, fabsf(q.s));
    }
    v = block_reduce(v, reinterpret_cast<Pair*>(scratch_raw));
    a = block_reduce(a, reinterpret_cast<float*>(scratch_raw));
    if (threadIdx.x == 0) {
        const double S = fabs((double)to_float(v));
        s_redo = p.fp64_auto && (double)p.units * 0x1p-48 * (double)a > 1e-6 * S;
    }
    __syncthreads();
    if (!s_redo) {
        if (threadIdx.x == 0) out_write(v, p);
        return;
    }
    double d = 0.0;
    for (int i = threadIdx.x; i < p.units; i += blockDim.x)
        d = __dadd_rn(d, to_double(slot_load<Pair>(p.partials + (size_t)i * 16)));
    d = block_reduce(d, reinterpret_cast<double*>(scratch_raw));
    if (threadIdx.x == 0) *reinterpret_cast<float*>(p.out) = __double2float_rn(__dmul_rn(d, (double)p.scale));
}

template <class A> __device__ __forceinline__ void reduce_slots_any(const KParams& p) {
    if (p.fp64) reduce_slots<double>(p);
    else reduce_slots<A>(p);
}
template <> __device__ __forceinline__ void reduce_slots_any<long long>(const KParams& p) {
    reduce_slots<long long>(p);
}

template <class A> __device__ __forceinline__ void store_unit(const KParams& p, int unit, A v) {
    unsigned char* slot = p.partials + (size_t)unit * 16;
    if (p.fp64) slot_store<double>(slot, to_double(v));
    else slot_store<A>(slot, v);
}
template <> __device__ __forceinline__ void store_unit<long long>(const KParams& p, int unit, long long v) {
    slot_store<long long>(p.partials + (size_t)unit * 16, v);
}

template <class A> __device__ __forceinline__ void out_write_unit(A v, const KParams& p) {
    if (p.fp64) out_write(to_double(v), p);
    else out_write(v, p);
}
template <> __device__ __forceinline__ void out_write_unit<long long>(long long v, const KParams& p) {
    out_write(v, p);
}

template <class A> struct IsInt { static constexpr bool v = false; };
template <> struct IsInt<long long> { static constexpr bool v = true; };

// ------------------------------------------------------------- epilogue
// Block, cluster and grid stages.  Every thread of every CTA calls it.
template <class A> __device__ __forceinline__ void finish(A v, const KParams& p) {
    __shared__ __align__(16) unsigned char scratch_raw[32 * sizeof(A)];
    __shared__ __align__(16) unsigned char cluster_raw[16 * sizeof(A)];
    __shared__ int s_last;

    A unit_sum = block_reduce(v, reinterpret_cast<A*>(scratch_raw));  // thread 0

    if (p.log2c > 0) {
        cg::cluster_group cl = cg::this_cluster();
        const unsigned rank = cl.block_rank();
        A* slots = reinterpret_cast<A*>(cluster_raw);
        if (threadIdx.x == 0) {
            A* dst = cl.map_shared_rank(slots, 0);
            dst[rank] = unit_sum;
        }
        cl.sync();
        if (rank != 0) return;  // only rank 0's shared memory is read after the barrier
        if (threadIdx.x < 32) {
            A r = (int)threadIdx.x < (1 << p.log2c) ? slots[threadIdx.x] : Op<A>::zero();
            r = warp_reduce(r);
            if (threadIdx.x == 0) unit_sum = r;
        }
    }
    const int unit = (int)(blockIdx.x >> p.log2c);

    switch (p.stage) {
    case kStageSingle:
        if (threadIdx.x == 0) out_write_unit(unit_sum, p);
        return;
    case kStageAtomic:
        if (threadIdx.x == 0) out_atomic(unit_sum, p);
        return;
    case kStageTwoKernel:
        if (threadIdx.x == 0) store_unit(p, unit, unit_sum);
        return;
    case kStageLastBlock:
        if (threadIdx.x == 0) {
            store_unit(p, unit, unit_sum);
            __threadfence();
            const unsigned t = atomicAdd(p.ticket, 1u);
            s_last = (t == (unsigned)p.units - 1u);
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        reduce_slots_any<A>(p);
        if (threadIdx.x == 0) atomicExch(p.ticket, 0u);  // ready for the next launch
        return;
    case kStageGridSync: {
        cg::grid_group g = cg::this_grid();
        if (!g.is_valid()) {  // not launched cooperatively: never wait
            if (threadIdx.x == 0) atomicOr(p.err, kErrNotCooperative);
            return;
        }
        if (threadIdx.x == 0) store_unit(p, unit, unit_sum);
        g.sync();
        if (blockIdx.x == 0) reduce_slots_any<A>(p);
        return;
    }
    default:
        return;
    }
}

// ------------------------------------------------------------ LDG path
template <int DT, bool COMP, int VB, int UNROLL>
__global__ void __launch_bounds__(1024) reduce_ldg_kernel(const KParams p) {
    using A = typename Acc<DT, COMP>::T;
    constexpr int W = VB / 4;
    grid_dependency_wait();
    allow_dependents();
    A acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = Op<A>::zero();
    Levels<A> lv;
    lv.init();

    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const unsigned char* body = p.x + p.head * ElemBytes<DT>::v;

    int64_t i = tid;
    if constexpr (std::is_same<A, float>::value) {
        // blocked (Levels<float>).  Unrolling factors: the compiler's own
        // choice for the block bookkeeping costs 10-25 registers on the
        // 16-byte shapes that run many CTAs per SM, so those are unrolled by
        // hand only (x2 for one load per iteration); the 32 B x 2 shape, which
        // serves inputs up to 16 MiB where a thread makes a few iterations,
        // is unrolled x4 so that their loads overlap (2^18 elements in one
        // cluster: 3.2 us with no unrolling, 2.45 us with it)
#pragma unroll (UNROLL == 1 ? 2 : (VB == 32 && UNROLL == 2 ? 4 : 1))
        for (; i + (UNROLL - 1) * nth < p.nvec; i += UNROLL * nth) {
            uint32_t v[UNROLL][W];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) ldg_vec(body + (i + u * nth) * VB, v[u]);
            AccBatch<DT, A, W, UNROLL>::run(acc, v);
            lv.template after<UNROLL * AddsPerWord<DT>::v>(acc);
        }
        for (; i < p.nvec; i += nth) {
            uint32_t v[W];
            ldg_vec(body + i * VB, v);
            AccVec<DT, A, W>::run(acc, v);
            lv.template after<AddsPerWord<DT>::v>(acc);
        }
    } else {
        for (; i + (UNROLL - 1) * nth < p.nvec; i += UNROLL * nth) {
            uint32_t v[UNROLL][W];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) ldg_vec(body + (i + u * nth) * VB, v[u]);
            AccBatch<DT, A, W, UNROLL>::run(acc, v);
        }
        for (; i < p.nvec; i += nth) {
            uint32_t v[W];
            ldg_vec(body + i * VB, v);
            AccVec<DT, A, W>::run(acc, v);
        }
    }
    if (tid < p.head) acc_elem<DT>(acc[0], p.x, tid);
    if (tid < p.ntail) acc_elem<DT>(acc[0], p.x, p.tail_begin + tid);

    A t = lv.total(acc);
    finish(t, p);
}

// ----------------------------------------------------------- BULK path
// Warp 0 lane 0 is the producer: it streams this CTA's tiles (tile k of the
// CTA is global tile blockIdx.x + k * gridDim.x) into a ring of `stages`
// shared-memory buffers with cp.async.bulk; warps 1.. consume.  full[s]
// completes when the copy of a tile into stage s has landed; empty[s] when
// every consumer warp is done with it.
template <int DT, bool COMP>
__global__ void __launch_bounds__(1024) reduce_bulk_kernel(const KParams p) {
    using A = typename Acc<DT, COMP>::T;
    extern __shared__ __align__(128) unsigned char dsm[];
    const int S = p.stages;
    const uint32_t ring = smem_u32(dsm);
    const uint32_t full0 = ring + (uint32_t)S * (uint32_t)p.tile_bytes;  // S mbarriers
    const uint32_t empty0 = full0 + 8u * S;                             // S mbarriers
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncw = (blockDim.x >> 5) - 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8u * s, 1);
            mbar_init(empty0 + 8u * s, (uint32_t)ncw);
        }
        mbar_fence_init();
    }
    grid_dependency_wait();  // shared-memory set-up above overlaps the previous kernel
    allow_dependents();
    __syncthreads();

    const int64_t my_tiles = p.ntiles > (int64_t)blockIdx.x
                                 ? (p.ntiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1
                                 : 0;
    const unsigned char* body = p.x + p.head * ElemBytes<DT>::v;
    A acc[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) acc[w] = Op<A>::zero();
    Levels<A> lv;
    lv.init();

    if (warp == 0) {
        if (lane == 0) {
            int64_t k = 0;
            bool ok = true;
            for (; k < my_tiles; ++k) {
                const int s = (int)(k % S);
                const uint32_t ph = (uint32_t)((k / S) & 1);
                if (k >= S && !mbar_wait_bounded(empty0 + 8u * s, ph ^ 1u, p.limit_ns)) {
                    atomicOr(p.err, kErrTimeout);
                    ok = false;
                    break;
                }
                const int64_t t = (int64_t)blockIdx.x + k * gridDim.x;
                const int64_t off = t * p.tile_bytes;
                const uint32_t bytes = (uint32_t)min((int64_t)p.tile_bytes, p.body_bytes - off);
                mbar_arrive_expect_tx(full0 + 8u * s, bytes);
                bulk_g2s(ring + (uint32_t)s * p.tile_bytes, body + off, bytes, full0 + 8u * s);
            }
            if (!ok) {
                // Do not leave while copies may still be writing this CTA's
                // shared memory: wait for the last one issued into each stage,
                // bounded separately (at least 1 s, whatever the spin limit).
                const uint64_t drain = p.limit_ns > 1000000000ull ? p.limit_ns : 1000000000ull;
                for (int64_t j = k - 1; j >= 0 && j >= k - S; --j) {
                    const int s = (int)(j % S);
                    mbar_wait_bounded(full0 + 8u * s, (uint32_t)((j / S) & 1), drain);
                }
            }
        }
    } else {
        const int ctid = threadIdx.x - 32, nct = ncw * 32;
        const int tile_chunks = p.tile_bytes >> 4;
        const int q_full = ctid < tile_chunks ? (tile_chunks - 1 - ctid) / nct + 1 : 0;
        (void)q_full;
        bool pending = false;  // float: acc holds a block to fold
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int s = (int)(k % S);
            const uint32_t ph = (uint32_t)((k / S) & 1);
            // one decision per warp: every lane leaves, or none does, so the
            // __syncwarp and the shuffles below always see the whole warp
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(full0 + 8u * s, ph, p.limit_ns))) {
                if (lane == 0) atomicOr(p.err, kErrTimeout);
                break;
            }
            const int64_t t = (int64_t)blockIdx.x + k * gridDim.x;
            const int chunks = (int)(min((int64_t)p.tile_bytes, p.body_bytes - t * p.tile_bytes) >> 4);
            const uint32_t base = ring + (uint32_t)s * p.tile_bytes;
            if constexpr (std::is_same<A, float>::value) {
                // This thread's q chunks of the tile form one block (at most
                // kChunks: kBlockAdds additions into each word), folded after
                // the stage is released; more chunks than that per tile are
                // split into blocks of kChunks.
                constexpr int kChunks = kBlockAdds / AddsPerWord<DT>::v;
                const int q = chunks == tile_chunks ? q_full
                                                    : (ctid < chunks ? (chunks - 1 - ctid) / nct + 1 : 0);
                if (q <= kChunks) {
                    int j = ctid;
                    for (; j + nct < chunks; j += 2 * nct) {
                        uint32_t v0[4], v1[4];
                        lds_vec(base + 16u * j, v0);
                        lds_vec(base + 16u * (j + nct), v1);
                        AccVec<DT, A, 4>::run(acc, v0);
                        AccVec<DT, A, 4>::run(acc, v1);
                    }
                    if (j < chunks) {
                        uint32_t v0[4];
                        lds_vec(base + 16u * j, v0);
                        AccVec<DT, A, 4>::run(acc, v0);
                    }
                } else {
                    int j = ctid;
                    for (int done = 0; done < q; done += kChunks) {
                        if (done) lv.flush(acc);
                        const int nb = q - done < kChunks ? q - done : kChunks;
                        int c = 0;
                        for (; c + 1 < nb; c += 2, j += 2 * nct) {
                            uint32_t v0[4], v1[4];
                            lds_vec(base + 16u * j, v0);
                            lds_vec(base + 16u * (j + nct), v1);
                            AccVec<DT, A, 4>::run(acc, v0);
                            AccVec<DT, A, 4>::run(acc, v1);
                        }
                        if (c < nb) {
                            uint32_t v0[4];
                            lds_vec(base + 16u * j, v0);
                            AccVec<DT, A, 4>::run(acc, v0);
                            j += nct;
                        }
                    }
                }
                pending = q > 0;
            } else {
                int j = ctid;
                for (; j + nct < chunks; j += 2 * nct) {
                    uint32_t v0[4], v1[4];
                    lds_vec(base + 16u * j, v0);
                    lds_vec(base + 16u * (j + nct), v1);
                    AccVec<DT, A, 4>::run(acc, v0);
                    AccVec<DT, A, 4>::run(acc, v1);
                }
                for (; j < chunks; j += nct) {
                    uint32_t v0[4];
                    lds_vec(base + 16u * j, v0);
                    AccVec<DT, A, 4>::run(acc, v0);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8u * s);
            if (pending) lv.flush(acc);
        }
        const int64_t gct = (int64_t)blockIdx.x * nct + ctid;
        if (gct < p.head) acc_elem<DT>(acc[0], p.x, gct);
        if (gct < p.ntail) acc_elem<DT>(acc[0], p.x, p.tail_begin + gct);
    }

    A t = lv.total(acc);
    finish(t, p);
}

// ---------------------------------------------- two-kernel second stage
template <class P> __global__ void __launch_bounds__(1024) reduce_final_kernel(const KParams p) {
    grid_dependency_wait();  // the implicit barrier: every unit's partial is written
    allow_dependents();
    reduce_slots<P>(p);
}

// ----------------------------------------------------- kernel selection
template <int DT, bool COMP, int VB>
inline const void* pick_ldg(int unroll) {
    switch (unroll) {
    case 1: return (const void*)reduce_ldg_kernel<DT, COMP, VB, 1>;
    case 2: return (const void*)reduce_ldg_kernel<DT, COMP, VB, 2>;
    case 4: return (const void*)reduce_ldg_kernel<DT, COMP, VB, 4>;
    case 8: return (const void*)reduce_ldg_kernel<DT, COMP, VB, 8>;
    default: return nullptr;
    }
}

template <int DT, bool COMP>
inline bool pick_kernels(bool fp64, bool bulk, int vec, int unroll, KernelSet* k) {
    using A = typename Acc<DT, COMP>::T;
    if (bulk) k->main = (const void*)reduce_bulk_kernel<DT, COMP>;
    else if (vec == 16) k->main = pick_ldg<DT, COMP, 16>(unroll);
    else if (vec == 32) k->main = pick_ldg<DT, COMP, 32>(unroll);
    else k->main = nullptr;
    if (IsInt<A>::v || !fp64) k->final = (const void*)reduce_final_kernel<A>;
    else k->final = (const void*)reduce_final_kernel<double>;
    return k->main != nullptr;
}

}  // namespace sr
