// Teams of CTAs that cooperate on one solve inside the persistent cooperative
// launch: a bounded-wait barrier, deterministic all-reductions of FP64
// partial sums, and the partition of element ranges among the team's CTAs.
#pragma once

#include "common.cuh"

namespace fde {

// ~2 s at GB300 clocks.  A barrier that waits longer records FDE_ETIMEOUT in
// the launch's abort flag; CTAs waiting at any barrier see the flag on their
// next poll and every CTA of the launch winds down.
constexpr long long kBarrierCycles = 4000000000LL;

struct Team {
    int rank;              // CTA index inside the team
    int size;              // CTAs in the team
    unsigned int* count;
    unsigned int* gen;
    double* partial;       // [size][kMaxDots]
    unsigned int* abort_flag;
    SyncArea* sync;
};

// Phase timestamps for performance analysis (compiled in with -DFDE_TRACE):
// CTA 0 of the launch appends (code, %globaltimer) pairs to the sync area.
FDE_D void trace_mark(const Team& t, int code) {
#ifdef FDE_TRACE
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long ns;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
        const unsigned int i = atomicAdd(&t.sync->trace_n, 1u);
        if (i < (unsigned)kTraceEntries) t.sync->trace[i] = ((unsigned long long)code << 48) | (ns & 0xffffffffffffULL);
    }
#else
    (void)t;
    (void)code;
#endif
}

// GPU-scope acquire load, release add and acquire-release add (PTX memory
// model): a CTA's writes before its arrival reach every CTA that observes the
// barrier's release, without full fences.
FDE_D unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
FDE_D unsigned int atom_add_acq_rel_gpu(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
FDE_D void atom_add_release_gpu(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    (void)old;
}

// Returns false when the launch is being aborted (a barrier timed out).
FDE_D bool team_sync(const Team& t, long long bound = kBarrierCycles) {
    __shared__ int s_ok;
    if (t.size == 1) {
        __syncthreads();
        return true;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // The CTA's writes precede this thread's release through the CTA
        // barrier above (releases are cumulative).  Arrivals form a release
        // sequence on the counter that the last arrival acquires; its release
        // of the generation is acquired by every waiting CTA.
        int ok = 1;
        const unsigned int g = ld_acquire_gpu(t.gen);
        const unsigned int arrived = atom_add_acq_rel_gpu(t.count, 1u);
        if (arrived == (unsigned int)t.size - 1u) {
            atomicExch(t.count, 0u);
            atom_add_release_gpu(t.gen, 1u);
        } else {
            // wait for the release of this generation; give up when the bound
            // runs out (and raise the launch's abort flag) or when another
            // team's barrier already has, so every CTA winds down within one
            // poll of the first timeout
            const long long t0 = clock64();
            while (ld_acquire_gpu(t.gen) == g) {
                if (ld_acquire_gpu(t.abort_flag) != 0u) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > bound) {
                    ok = 0;
                    atomicExch(t.abort_flag, 1u);
                    break;
                }
            }
        }
        s_ok = ok && (ld_acquire_gpu(t.abort_flag) == 0u);
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename R>
FDE_D R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sums of K per-thread values (K <= blockDim/32), written to
// out[0..K) in shared memory.  The values are transposed through `wide`
// (K * blockDim doubles of shared memory) and warp k sums column k: lane l
// adds entries l, l+32, ... in order, then a fixed shuffle tree.  Each sum
// costs blockDim/32 + 5 warp-wide FP64 adds instead of 5 per warp, which
// matters where every FP64 warp instruction occupies the SM's FP64 pipe for
// many cycles.  Deterministic.
template <int K>
FDE_D void block_sum(const double (&v)[K], double* out, double* wide) {
    const int nt = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) wide[k * nt + threadIdx.x] = v[k];
    __syncthreads();
    if (warp < K) {
        // four interleaved partial sums, then a fixed tree: short dependency
        // chains (a dependent FP64 add is slow here), still one fixed order
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        int u = 0;
        for (int i = lane; i < nt; i += 32, u = (u + 1) & 3) a[u] += wide[warp * nt + i];
        double s = (a[0] + a[1]) + (a[2] + a[3]);
        s = warp_sum(s);
        if (lane == 0) out[warp] = s;
    }
    __syncthreads();
}

// Compensated FP32 accumulation (for FP32 vectors): the product a*b is split
// exactly into p + e with one FMA, the running sum s absorbs p through an
// error-free TwoSum, and both rounding errors collect in c.  (s + c) carries
// roughly twice the FP32 precision -- FP64-class inner products without the
// FP64 pipe, which on this GPU issues at a small fraction of the FP32 rate.
struct F2 {
    float s, c;
};

FDE_D void two_sum_acc(F2& a, float p) {
    const float t = a.s + p;
    const float bp = t - a.s;
    a.c += (a.s - (t - bp)) + (p - bp);
    a.s = t;
}

FDE_D void dot2_acc(F2& a, float x, float y) {
    const float p = x * y;
    const float e = fmaf(x, y, -p);
    two_sum_acc(a, p);
    a.c += e;
}

// Block-wide sums of K compensated FP32 values, transposed through `wide`
// (K * blockDim float pairs) like block_sum; warp k accumulates column k with
// TwoSum, then a shuffle tree of compensated adds.  out[0..K) in FP64.
template <int K>
FDE_D void block_sum_f2(const F2 (&v)[K], double* out, double* wide) {
    float2* w2 = reinterpret_cast<float2*>(wide);
    const int nt = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) w2[k * nt + threadIdx.x] = make_float2(v[k].s, v[k].c);
    __syncthreads();
    if (warp < K) {
        F2 a{0.0f, 0.0f};
        for (int i = lane; i < nt; i += 32) {
            const float2 e = w2[warp * nt + i];
            two_sum_acc(a, e.x);
            a.c += e.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, a.s, o);
            const float oc = __shfl_xor_sync(0xffffffffu, a.c, o);
            two_sum_acc(a, os);
            a.c += oc;
        }
        if (lane == 0) out[warp] = (double)a.s + (double)a.c;
    }
    __syncthreads();
}

// vals[0..K) (shared memory, this CTA's totals) -> team totals in every CTA.
FDE_D bool team_allreduce(const Team& t, double* vals, int K) {
    if (t.size == 1) return true;
    for (int k = threadIdx.x; k < K; k += blockDim.x) t.partial[t.rank * kMaxDots + k] = vals[k];
    if (!team_sync(t)) return false;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int k = warp; k < K; k += nw) {
        double s = 0.0;
        for (int r = lane; r < t.size; r += 32) s += __ldcg(t.partial + r * kMaxDots + k);
        s = warp_sum(s);
        if (lane == 0) vals[k] = s;
    }
    __syncthreads();
    return true;
}

// [lo, hi) of an N-element vector owned by this CTA for elementwise phases.
FDE_D void team_range(const Team& t, long long N, long long& lo, long long& hi) {
    long long chunk = (N + t.size - 1) / t.size;
    chunk = (chunk + 255) & ~255LL;
    lo = (long long)t.rank * chunk;
    hi = lo + chunk;
    if (hi > N) hi = N;
    if (lo > N) lo = N;
}

}  // namespace fde
