// The persistent cooperative kernel.  One launch runs a batch of independent
// solves (or one operator application): CTAs form teams; a team of one CTA
// pulls instances from a queue (largest first), a team of many CTAs works on
// one instance at a time with team barriers between phases.
#pragma once

#include "krylov.cuh"

namespace fde {

enum Op : int { kOpSolve = 0, kOpMatvec = 1, kOpTau = 2, kOpMatvecSub = 3 };   // kOpMatvecSub: out -= M in
enum Mode : int { kModeF64 = 0, kModeF32 = 1, kModeIR = 2 };

// Products with M one inner FP32 PCG solve of the refinement mode may take.
constexpr int kInnerPcgIters = 50;

struct EngineArgs {
    int op;
    int count;
    int team_size;             // team_mode 0: every team has team_size CTAs
    int team_mode;             // 1: team i = CTAs [sync->team_start[i], team_start[i+1]), instance i
    int dtype;                 // operator calls: FDE_F64 / FDE_F32
    int smem_bytes;            // dynamic shared memory of the launch
    SyncArea* sync;
    fde_solve_info* info;
    double tol, inner_tol;
    int max_iters, max_outer, side;
    const Inst* inst[kMaxBatch];
    const void* in[kMaxBatch];
    void* out[kMaxBatch];
    unsigned short order[kMaxBatch];
};

FDE_D int lm_f64(const Inst& I) { return I.line_mode & 0xff; }
FDE_D int lm_f32(const Inst& I) { return (I.line_mode >> 8) & 0xff; }

// FP64 residual r64 = b - A x and its norm (refinement and FP32 modes).
static FDE_NI bool residual64(const Team& t, const Inst& I, const double* b, const double* x, KShared& ks,
                              const Wk& wk, double& rn) {
    // r64 = b - A x, written by the matvec's epilogue (t64 is the 2D scratch)
    if (!op_matvec_out<double>(t, I, lm_f64(I), x, 1.0, I.t64, OutSpec<double>{kOutResid, I.r64, b}, wk))
        return false;
    const double* a[1] = {I.r64};
    if (!dots_pairs<double, 1>(t, I.N, a, a, ks)) return false;
    rn = sqrt(ks.red[0]);
    return true;
}

template <int MODE>
FDE_D bool run_solve(const Team& t, const Inst& I, const EngineArgs& a, int idx, KShared& ks, const Wk& wk) {
    const double* b = reinterpret_cast<const double*>(a.in[idx]);
    double* x = reinterpret_cast<double*>(a.out[idx]);
    SolveState st{};
    st.status = FDE_ENOCONV;
    int outer = 0;
    int res64 = 0;             // FP64 residuals of the refinement and FP32 modes
    int its64 = 0;             // iterations on FP64 vectors (FP64 mode: all; refinement: an FP64 finish)
    const long long N = I.N;
    long long lo, hi;
    team_range(t, N, lo, hi);
    if constexpr (MODE == kModeF64) {
        SolveParams sp{a.tol, a.max_iters, a.side, 0};
        if (!krylov_core<double>(t, I, lm_f64(I), b, x, sp, st, ks, wk)) return false;
        its64 = st.iterations;
    } else {
        float* rhs32 = reinterpret_cast<float*>(I.wvec) + extra_vec_offset<float>(I);
        float* sol32 = rhs32 + N;
        {
            const double* p[1] = {b};
            if (!dots_pairs<double, 1>(t, N, p, p, ks)) return false;
        }
        const double nb = sqrt(ks.red[0]);
        if constexpr (MODE == kModeF32) {
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                rhs32[i] = float(__ldcg(b + i));
                sol32[i] = float(x[i]);
            }
            if (!team_sync(t)) return false;
            SolveParams sp{a.tol, a.max_iters, a.side, 1};
            if (!krylov_core<float>(t, I, lm_f32(I), rhs32, sol32, sp, st, ks, wk)) return false;
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) x[i] = double(sol32[i]);
            if (!team_sync(t)) return false;
            double rn;
            if (!residual64(t, I, b, x, ks, wk, rn)) return false;
            ++res64;
            st.relres = nb > 0.0 ? rn / nb : 0.0;
            if (st.status == FDE_OK && !(st.relres <= a.tol)) st.status = FDE_ENOCONV;
        } else {
            int status = FDE_ENOCONV;
            int inner_status = FDE_OK;
            double rn_prev = 0.0;
            while (true) {
                double rn;
                if (!residual64(t, I, b, x, ks, wk, rn)) return false;
                ++res64;
                st.relres = nb > 0.0 ? rn / nb : 0.0;
                if (!finite(rn)) { status = FDE_ENONFINITE; break; }
                if (rn <= a.tol * nb) { status = FDE_OK; break; }
                if (outer >= a.max_outer || st.iterations >= a.max_iters) { status = FDE_ENOCONV; break; }
                if (inner_status == FDE_EBREAKDOWN || inner_status == FDE_ENONFINITE) { status = inner_status; break; }
                if (outer >= 1 && rn > 0.25 * rn_prev) {
                    // A correction shrank the FP64 residual less than fourfold: the
                    // FP32 operator does not resolve the error (kappa(M) u32 log2 L is
                    // not small).  Finish this solve in FP64 from the current x.
                    SolveState s64{};
                    s64.iterations = st.iterations;
                    SolveParams sp{a.tol, a.max_iters, a.side, 0};
                    if (!krylov_core<double>(t, I, lm_f64(I), b, x, sp, s64, ks, wk)) return false;
                    its64 = s64.iterations - st.iterations;
                    st.iterations = s64.iterations;
                    st.restarts += s64.restarts;
                    st.basis_sum += s64.basis_sum;
                    st.reorth += s64.reorth;
                    st.cycles += s64.cycles;
                    st.relres = s64.relres;
                    st.relres_est = s64.relres_est;
                    status = s64.status;
                    break;
                }
                rn_prev = rn;
                const double inv = 1.0 / rn;
                for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                    rhs32[i] = float(I.r64[i] * inv);
                    sol32[i] = 0.0f;
                }
                if (!team_sync(t)) return false;
                SolveState in{};
                in.iterations = st.iterations;
                // An FP32 solve that has not reached inner_tol within two restart
                // cycles is limited by FP32 resolution, not by the Krylov space: more
                // iterations only chase rounding noise (about 900 for alpha = 1.8 at
                // n = 65535).  Its correction goes to the contraction test above.
                const int cap = st.iterations + (I.method == FDE_GMRES ? 2 * I.restart : kInnerPcgIters);
                // A residual already within a modest factor of the target needs a
                // correction that closes only that gap (with a margin of 3): solving
                // it to inner_tol spends iterations on accuracy the refinement
                // discards.  At most a halving is asked of any correction.
                double itol = a.inner_tol;
                const double need = 0.3 * a.tol * nb / rn;
                if (need > itol) itol = need < 0.5 ? need : 0.5;
                SolveParams sp{itol, cap < a.max_iters ? cap : a.max_iters, a.side, 1};
                if (!krylov_core<float>(t, I, lm_f32(I), rhs32, sol32, sp, in, ks, wk)) return false;
                st.iterations = in.iterations;
                st.restarts += in.restarts;
                st.basis_sum += in.basis_sum;
                st.reorth += in.reorth;
                st.cycles += in.cycles;
                st.relres_est = in.relres_est;
                inner_status = in.status;
                for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) x[i] = x[i] + rn * double(sol32[i]);
                if (!team_sync(t)) return false;
                ++outer;
            }
            st.status = status;
        }
    }
    if (t.rank == 0 && threadIdx.x == 0) {
        fde_solve_info inf;
        inf.status = st.status;
        inf.iterations = st.iterations;
        inf.outer = outer;
        inf.restarts = st.restarts;
        inf.relres = st.relres;
        inf.relres_est = st.relres_est;
        inf.basis_sum = st.basis_sum;
        inf.reorth = st.reorth;
        inf.cycles = st.cycles;
        inf.residuals64 = res64;
        inf.iterations64 = its64;
        inf.reserved = 0;
        a.info[idx] = inf;
    }
    return true;
}

template <int MODE>
FDE_D bool run_op(const Team& t, const Inst& I, const EngineArgs& a, int idx, const Wk& wk) {
    const bool f64 = (MODE == kModeF64) || a.dtype == FDE_F64;
    if (f64) {
        const double* in = reinterpret_cast<const double*>(a.in[idx]);
        double* out = reinterpret_cast<double*>(a.out[idx]);
        if (a.op == kOpMatvec) return op_matvec<double>(t, I, lm_f64(I), in, 1.0, out, I.t64, wk);
        if (a.op == kOpMatvecSub)
            return op_matvec_out<double>(t, I, lm_f64(I), in, 1.0, I.t64, OutSpec<double>{kOutResid, out, out}, wk);
        return op_tau<double>(t, I, lm_f64(I), in, 1.0, out, wk);
    }
    if constexpr (MODE != kModeF64) {
        const float* in = reinterpret_cast<const float*>(a.in[idx]);
        float* out = reinterpret_cast<float*>(a.out[idx]);
        float* tmp = reinterpret_cast<float*>(I.t64);
        if (a.op == kOpMatvec) return op_matvec<float>(t, I, lm_f32(I), in, 1.0f, out, tmp, wk);
        if (a.op == kOpMatvecSub)
            return op_matvec_out<float>(t, I, lm_f32(I), in, 1.0f, tmp, OutSpec<float>{kOutResid, out, out}, wk);
        return op_tau<float>(t, I, lm_f32(I), in, 1.0f, out, wk);
    }
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) fde_engine(const __grid_constant__ EngineArgs a) {
    extern __shared__ __align__(256) unsigned char dsm[];
    __shared__ Inst s_inst;
    __shared__ unsigned int s_next;
    int ts, nteams, team_id, first;
    if (a.team_mode == 1) {
        // sizes written by k_balance earlier on the stream
        const unsigned short* st = a.sync->team_start;
        nteams = a.count;
        team_id = -1;
        for (int i = 0; i < nteams; ++i)
            if ((int)blockIdx.x >= st[i] && (int)blockIdx.x < st[i + 1]) { team_id = i; break; }
        if (team_id < 0) return;
        first = st[team_id];
        ts = st[team_id + 1] - first;
    } else {
        ts = a.team_size;
        nteams = gridDim.x / ts;
        team_id = blockIdx.x / ts;
        if (team_id >= nteams) return;
        first = team_id * ts;
    }
    // per-CTA constants in shared memory: functions reach them through
    // references, which for a thread-local object would be stack (local
    // memory) loads that miss the small L1 left beside the work area
    __shared__ Team s_team;
    __shared__ Wk s_wk;
    __shared__ KShared s_ks;
    if (threadIdx.x == 0) {
        s_team.rank = blockIdx.x - first;
        s_team.size = ts;
        s_team.count = &a.sync->bar_count[team_id];
        s_team.gen = &a.sync->bar_gen[team_id];
        s_team.partial = a.sync->partial + (size_t)first * kMaxDots;
        s_team.abort_flag = &a.sync->abort_flag;
        s_team.sync = a.sync;
    }
    __syncthreads();
    const Team& t = s_team;
    int next_static = team_id;
    while (true) {
        int idx;
        if (ts == 1) {
            if (threadIdx.x == 0) s_next = atomicAdd(&a.sync->queue, 1u);
            __syncthreads();
            idx = (int)s_next;
            __syncthreads();
        } else {
            idx = next_static;
            next_static += nteams;
        }
        if (idx >= a.count) break;
        if (*reinterpret_cast<volatile unsigned int*>(&a.sync->abort_flag)) break;
        const int inst_i = a.team_mode == 1 ? idx : a.order[idx];
        {
            const int* src = reinterpret_cast<const int*>(a.inst[inst_i]);
            int* dst = reinterpret_cast<int*>(&s_inst);
            for (int w = threadIdx.x; w < (int)(sizeof(Inst) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
        }
        __syncthreads();
        const int m = s_inst.method == FDE_GMRES ? s_inst.restart : 1;
        const size_t hdr = kshared_bytes(m, s_inst.logTsm);
        if (threadIdx.x == 0) {
            KShared k = kshared_carve(dsm, m);
            k.wide = reinterpret_cast<double*>(dsm + hdr);
            k.twq32 = reinterpret_cast<cx<float>*>(k.twq + padded_len((1 << s_inst.logTsm) >> 2));
            s_ks = k;
            s_wk.smem = dsm + hdr;
            s_wk.bytes = a.smem_bytes - (int)hdr;
            s_wk.tw.q = k.twq;
            s_wk.tw.q32 = k.twq32;
            s_wk.tw.logT = s_inst.logTsm;
            s_wk.tw.g64 = s_inst.tw64;
            s_wk.tw.g32 = s_inst.tw32;
            s_wk.tw.logTW = s_inst.logTW;
        }
        __syncthreads();
        KShared& ks = s_ks;
        const Wk& wk = s_wk;
        // quarter-wave twiddle table of W_T, T = 2^logTsm, from the global table;
        // entry i at pad(i), so the strided lookups of the later radix passes
        // (index r k 2^s) spread over the banks
        {
            const int q = (1 << s_inst.logTsm) >> 2;
            const int sh = s_inst.logTW - s_inst.logTsm;
            for (int i = threadIdx.x; i < q; i += blockDim.x) {
                const cx<double> w = s_inst.tw64[i << sh];
                ks.twq[pad(i)] = w;
                ks.twq32[pad(i)] = mk((float)w.x, (float)w.y);
            }
        }
        __syncthreads();
        bool ok;
        if (a.op == kOpSolve) ok = run_solve<MODE>(t, s_inst, a, inst_i, ks, wk);
        else ok = run_op<MODE>(t, s_inst, a, inst_i, wk);
        if (!ok) {
            if (threadIdx.x == 0 && t.rank == 0 && a.op == kOpSolve) {
                a.info[inst_i].status = FDE_ETIMEOUT;
            }
            break;
        }
        __syncthreads();
    }
}

}  // namespace fde
