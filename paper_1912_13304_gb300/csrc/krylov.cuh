// Device-resident Krylov drivers: PCG and restarted GMRES(m) (right or left
// preconditioned), and the FP32-inner / FP64-outer iterative refinement
// around them.  Every CTA of a team runs the same scalar recurrences on the
// same deterministic reductions, so all CTAs take identical decisions
// without extra barriers.  Inner products, norms, the Hessenberg matrix and
// the Givens rotations are FP64 whatever the vector precision.
//
// Right-preconditioned GMRES uses a fused Arnoldi step: the basis vector
// v_j = w_{j-1} - sum_q c_q v_q is formed on the fly by the first transform
// phase of the tau solve (and stored there), the tau solve hands z straight
// to the matvec on the same CTAs where the layout allows, and the matvec's
// last phase is followed by the partial inner products <w, v_i> and ||w||^2
// of the elements the CTA produced -- one reduction per iteration.
// Classical Gram-Schmidt is reorthogonalised (a second pass) only when the
// projection leaves less than ||w|| / sqrt(2) (the Daniel-Gragg-Kaufman-
// Stewart test).  For FP32
// vectors the Gram-Schmidt inner products sum each thread's elements in FP32
// (FMA) and the block and team partials in FP64; PCG's scalar products and the
// right-hand side norms use compensated FP32 arithmetic (team.cuh).  A
// compensated term costs about ten instructions, which made the basis passes
// of the 2D inner solves instruction-bound.
#pragma once

#include "ops.cuh"

namespace fde {

struct SolveParams {
    double tol;            // relative to ||rhs||
    int max_iters;         // cap on products with M
    int side;              // FDE_SIDE_RIGHT / FDE_SIDE_LEFT
    int inner;             // inner solve of a refinement: stop on the Krylov estimate
};

struct SolveState {
    int iterations;
    int restarts;
    int status;
    double relres_est;
    double relres;         // true residual of the last check, relative to ||rhs||
    // work counters (fde_solve_info): sum over Arnoldi steps of the basis
    // vectors each step orthogonalised against, second Gram-Schmidt passes,
    // Krylov cycles started from a true residual
    int basis_sum;
    int reorth;
    int cycles;
};

// Shared-memory scalars of one CTA (identical in every CTA of a team), and
// the quarter-wave twiddle table.
struct KShared {
    double* H;             // (m+1) x m, column-major H[i + j (m+1)]
    double* cs;
    double* sn;
    double* g;
    double* y;
    double* vs;            // 1/||v_i|| of the stored (unnormalised) basis vectors
    double* red;           // reduction results, kMaxDots
    double* sc;            // 8 scalars that thread 0 computes for the CTA (red + kMaxDots)
    double* wide;          // block_sum transpose area: the transform work area, idle during reductions
    double* coef;          // coefficients of the next on-the-fly basis vector
    float* coef32;         // the same, for FP32 vectors
    cx<double>* twq;       // W_T^t, t < T/4
    cx<float>* twq32;
};

// Coefficients in the working precision.
template <typename W> FDE_D W* kcoef(KShared& ks);
template <> FDE_D double* kcoef<double>(KShared& ks) { return ks.coef; }
template <> FDE_D float* kcoef<float>(KShared& ks) { return ks.coef32; }
// Thread 0 sets coefficient q in both precisions.
FDE_D void set_coef(KShared& ks, int q, double v) {
    ks.coef[q] = v;
    ks.coef32[q] = (float)v;
}

FDE_HD size_t kshared_scalar_bytes(int m) {
    const size_t d = (size_t)(m + 1) * m + 3 * (size_t)m + 2 * (size_t)(m + 2) + (kMaxDots + 8) + 8 * 32 +
                     (kMaxDots + 2) + (kMaxDots + 2) / 2 + 1;
    return ((d * sizeof(double)) + 255) & ~(size_t)255;
}

// Rounded to 256 bytes: the transform buffers that follow need 16-byte
// alignment whatever the table size.
FDE_HD size_t kshared_bytes(int m, int logT) {
    // the quarter-wave tables are padded like the line buffers (entry i at pad(i))
    const size_t b = kshared_scalar_bytes(m) + (size_t)padded_len((1 << logT) / 4) * (sizeof(cx<double>) + sizeof(cx<float>));
    return (b + 255) & ~(size_t)255;
}

FDE_D KShared kshared_carve(unsigned char* base, int m) {
    double* p = reinterpret_cast<double*>(base);
    KShared k;
    k.H = p; p += (m + 1) * m;
    k.cs = p; p += m;
    k.sn = p; p += m;
    k.y = p; p += m;
    k.g = p; p += m + 2;
    k.vs = p; p += m + 2;
    k.red = p; p += kMaxDots + 8;
    k.sc = k.red + kMaxDots;
    k.wide = nullptr;
    p += 8 * 32;
    k.coef = p; p += kMaxDots + 2;
    k.coef32 = reinterpret_cast<float*>(p);
    k.twq = reinterpret_cast<cx<double>*>(base + kshared_scalar_bytes(m));
    return k;
}

FDE_D bool finite(double v) { return isfinite(v); }

// sum_{q < n} v_q^2 by one thread with four interleaved accumulators (fixed order).
FDE_D double sum_squares(const double* v, int n) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < n; ++q) a[q & 3] += v[q] * v[q];
    return (a[0] + a[1]) + (a[2] + a[3]);
}

// ---------------------------------------------------------------------------
// Reductions over N-vectors
// ---------------------------------------------------------------------------

// ks.red[i] = <a, vs_i V_i> for i < cnt; with `norm`, ks.red[cnt] = <a, a>,
// summed over the elements that own(f) visits (f(p) per element, threads of
// this CTA), then over the team.
template <typename W, typename OwnF>
FDE_D bool dots_own(const Team& t, long long N, const W* a, const W* V, const double* vs, int cnt, bool norm,
                    KShared& ks, OwnF own) {
    const int tot = cnt + (norm ? 1 : 0);
    for (int c0 = 0; c0 < tot; c0 += 8) {
        if constexpr (sizeof(W) == 8) {
            double acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = 0.0;
            own([&](long long i) {
                const double ai = (double)ldw(a + i);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int kk = c0 + k;
                    if (kk < cnt) acc[k] += ai * (double)ldw(V + (long long)kk * N + i);
                    else if (kk == cnt && norm) acc[k] += ai * ai;
                }
            });
            block_sum<8>(acc, ks.red + c0, ks.wide);
        } else {
            // FP32 vectors of a Krylov basis: each thread sums its few elements in
            // FP32 (FMA), the block and team sums run in FP64
            float acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
            own([&](long long i) {
                const float ai = (float)ldw(a + i);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int kk = c0 + k;
                    if (kk < cnt) acc[k] = fmaf(ai, (float)ldw(V + (long long)kk * N + i), acc[k]);
                    else if (kk == cnt && norm) acc[k] = fmaf(ai, ai, acc[k]);
                }
            });
            double part[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) part[k] = acc[k];
            block_sum<8>(part, ks.red + c0, ks.wide);
        }
    }
    if (threadIdx.x < cnt) ks.red[threadIdx.x] *= vs[threadIdx.x];
    __syncthreads();
    trace_mark(t, 60);
    return team_allreduce(t, ks.red, tot);
}

// The same over the team's contiguous ranges: each thread keeps two elements'
// loads of 8 vectors in flight.
template <typename W>
FDE_D bool dots_basis(const Team& t, long long N, const W* a, const W* V, const double* vs, int cnt, bool norm,
                      KShared& ks) {
    long long lo, hi;
    team_range(t, N, lo, hi);
    const int tot = cnt + (norm ? 1 : 0);
    const int nt = blockDim.x;
    for (int c0 = 0; c0 < tot; c0 += 8) {
        if constexpr (sizeof(W) == 8) {
            double acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = 0.0;
            for (long long i0 = lo + threadIdx.x; i0 < hi; i0 += 2 * nt) {
                const long long i1 = i0 + nt;
                const bool h1 = i1 < hi;
                const double a0 = ldw(a + i0), a1 = h1 ? (double)ldw(a + i1) : 0.0;
                double v0[8], v1[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int kk = c0 + k;
                    v0[k] = kk < cnt ? (double)ldw(V + (long long)kk * N + i0) : a0;
                    v1[k] = kk < cnt ? (h1 ? (double)ldw(V + (long long)kk * N + i1) : 0.0) : a1;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (c0 + k < tot) acc[k] += a0 * v0[k] + a1 * v1[k];
            }
            block_sum<8>(acc, ks.red + c0, ks.wide);
        } else {
            // per-thread FP32 sums (FMA), FP64 block and team sums (see dots_own)
            float acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
            for (long long i0 = lo + threadIdx.x; i0 < hi; i0 += 2 * nt) {
                const long long i1 = i0 + nt;
                const bool h1 = i1 < hi;
                const float a0 = (float)ldw(a + i0), a1 = h1 ? (float)ldw(a + i1) : 0.0f;
                float v0[8], v1[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int kk = c0 + k;
                    v0[k] = kk < cnt ? (float)ldw(V + (long long)kk * N + i0) : a0;
                    v1[k] = kk < cnt ? (h1 ? (float)ldw(V + (long long)kk * N + i1) : 0.0f) : a1;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (c0 + k < tot) acc[k] = fmaf(a1, v1[k], fmaf(a0, v0[k], acc[k]));
            }
            double part[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) part[k] = acc[k];
            block_sum<8>(part, ks.red + c0, ks.wide);
        }
    }
    if (threadIdx.x < cnt) ks.red[threadIdx.x] *= vs[threadIdx.x];
    __syncthreads();
    trace_mark(t, 60);
    return team_allreduce(t, ks.red, tot);
}

// V_j = w - sum_{q < cnt} c_q V_q over this CTA's contiguous part of the team
// range, two elements and four vectors of loads in flight per thread.
template <typename W>
FDE_D void form_basis(const Team& t, long long N, const W* w, const W* V, const W* c, int cnt, W* out) {
    long long lo, hi;
    team_range(t, N, lo, hi);
    const int nt = blockDim.x;
    for (long long i0 = lo + threadIdx.x; i0 < hi; i0 += 2 * nt) {
        const long long i1 = i0 + nt;
        const bool h1 = i1 < hi;
        W a0 = ldw(w + i0), a1 = h1 ? ldw(w + i1) : W(0);
        int q = 0;
        for (; q + 4 <= cnt; q += 4) {
            W v0[4], v1[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                v0[r] = ldw(V + (long long)(q + r) * N + i0);
                v1[r] = h1 ? ldw(V + (long long)(q + r) * N + i1) : W(0);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                a0 -= c[q + r] * v0[r];
                a1 -= c[q + r] * v1[r];
            }
        }
        for (; q < cnt; ++q) {
            a0 -= c[q] * ldw(V + (long long)q * N + i0);
            if (h1) a1 -= c[q] * ldw(V + (long long)q * N + i1);
        }
        out[i0] = a0;
        if (h1) out[i1] = a1;
    }
}

// ks.red[k] = <a_k, b_k> for up to 8 pairs over the team partition.
template <typename W, int K>
FDE_D bool dots_pairs(const Team& t, long long N, const W* const (&a)[K], const W* const (&b)[K], KShared& ks) {
    long long lo, hi;
    team_range(t, N, lo, hi);
    if constexpr (sizeof(W) == 8) {
        double acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0.0;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] += (double)ldw(a[k] + i) * (double)ldw(b[k] + i);
        }
        block_sum<K>(acc, ks.red, ks.wide);
    } else {
        F2 acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = F2{0.0f, 0.0f};
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
#pragma unroll
            for (int k = 0; k < K; ++k) dot2_acc(acc[k], (float)ldw(a[k] + i), (float)ldw(b[k] + i));
        }
        block_sum_f2<K>(acc, ks.red, ks.wide);
    }
    return team_allreduce(t, ks.red, K);
}

// ---------------------------------------------------------------------------
// Fused right-preconditioned Arnoldi application:
//   z = P^{-1} u, w = M z, ks.red[i] = <w, vs_i V_i> (i < nd), ks.red[nd] = ||w||^2.
// ---------------------------------------------------------------------------

template <typename W>
FDE_NI bool arnoldi_right(const Team& t, const Inst& I, int lm, Combo<W> u, int nd, const W* V, W* z, W* w,
                          W* tmp, KShared& ks, const Wk& wk) {
    const long long N = I.N;
    const W* dinv = Prec<W>::dinv(I);
    const bool pre = I.has_D && I.order == FDE_ORDER_D_TAU;
    trace_mark(t, 20);
    if (I.order == FDE_ORDER_TRI) {
        // P_tri: the tridiagonal solve, then the matvec, then the dots
        if (!op_tau_combo<W>(t, I, lm, u, z, out_store<W>(z), wk)) return false;
        if (!op_matvec_out<W>(t, I, lm, z, W(1), tmp, out_store<W>(w), wk)) return false;
        return dots_basis<W>(t, N, w, V, ks.vs, nd, true, ks);
    }
    if (I.dim == 1 && lm == kLineCta) {
        // team of one: everything stays in this CTA
        cta_tau_1d<W>(I, wk, u, epi_a<W>(nullptr, out_store<W>(z)));
        cta_matvec_1d<W>(I, wk, z, W(1), epi_mvx<W>(I, z, W(1), out_store<W>(w)));
        trace_mark(t, 13);
        return dots_own<W>(t, N, w, V, ks.vs, nd, true, ks, [&](auto f) {
            for (long long i = threadIdx.x; i < N; i += blockDim.x) f(i);
        });
    }
    if (I.dim == 1) {
        const AxisData& A = I.ax[0];
        cx<W>* Y = Prec<W>::split(I);
        cx<W>* Y2 = Y + A.Np;
        const bool sym = I.symx;
        if (pre) u.pre = dinv;
        const int cc = split_cols_per_unit<W>(A, t.size, wk.bytes);
        split_fwd_cols<W, kExtOdd>(t, I, wk, u, Y, cc);
        if (!team_sync(t)) return false;
        trace_mark(t, 21);
        split_rows<W>(t, I, wk, mult_tau1<W>(A), Y, nullptr);
        if (!team_sync(t)) return false;
        trace_mark(t, 22);
        split_tau_inv_mv_fwd<W>(t, I, wk, Y, Y, cc, z);
        if (!team_sync(t)) return false;
        trace_mark(t, 11);
        split_rows<W>(t, I, wk, mult_matvec<W>(A, sym), Y, Y2);
        if (!team_sync(t)) return false;
        trace_mark(t, 12);
        split_inv_cols<W>(t, I, wk, Y, Y2, cc, !sym, epi_mvx<W>(I, z, W(1), out_store<W>(w)));
        trace_mark(t, 13);
        const int units = split_units(A, cc);
        return dots_own<W>(t, N, w, V, ks.vs, nd, true, ks, [&](auto f) {
            for (int un = t.rank; un < units; un += t.size)
                split_unit_elements(A, un * cc, split_width(A, un * cc, cc), f);
        });
    }
    // 2D plane: rows (first sine transform) | columns (tau) | rows (second sine
    // transform + x part of the matvec) | columns (y part) + dots
    if (pre) u.pre = dinv;
    plane_dst_rows<W>(t, I, wk, u, nullptr, z);
    if (!team_sync(t)) return false;
    trace_mark(t, 21);
    if (!plane_cols_tau<W>(t, I, wk, z)) return false;
    if (!team_sync(t)) return false;
    trace_mark(t, 22);
    plane_dst_matvec_rows<W>(t, I, wk, z, z, tmp);
    if (!team_sync(t)) return false;
    trace_mark(t, 11);
    if (!plane_cols_matvec<W>(t, I, wk, z, W(1), epi_mvy<W>(I, tmp, out_store<W>(w)))) return false;
    trace_mark(t, 13);
    // the column phase scatters each CTA's outputs over the plane: reduce over
    // contiguous ranges instead, once every CTA's part is written
    if (!team_sync(t)) return false;
    return dots_basis<W>(t, N, w, V, ks.vs, nd, true, ks);
}

// ---------------------------------------------------------------------------
// GMRES(m)
// ---------------------------------------------------------------------------

template <typename W>
struct GVecs {
    W* V;       // (m+1) N
    W* w;
    W* z;
    W* tt;
};

template <typename W>
FDE_D GVecs<W> gmres_vecs(const Inst& I) {
    W* b = reinterpret_cast<W*>(I.wvec);
    const long long N = I.N;
    const int m = I.restart;
    GVecs<W> v;
    v.V = b;
    v.w = b + (long long)(m + 1) * N;
    v.z = v.w + N;
    v.tt = v.z + N;
    return v;
}

template <typename W>
FDE_D long long extra_vec_offset(const Inst& I) {
    return I.method == FDE_GMRES ? (long long)(I.restart + 4) * I.N : 5LL * I.N;
}

// Givens rotation of Hessenberg column j (thread 0); updates g.
FDE_D void givens_column(KShared& ks, int j, int m) {
    double* Hc = ks.H + j * (m + 1);
    for (int q = 0; q < j; ++q) {
        const double a = ks.cs[q] * Hc[q] + ks.sn[q] * Hc[q + 1];
        Hc[q + 1] = -ks.sn[q] * Hc[q] + ks.cs[q] * Hc[q + 1];
        Hc[q] = a;
    }
    const double den = hypot(Hc[j], Hc[j + 1]);
    ks.cs[j] = den > 0.0 ? Hc[j] / den : 1.0;
    ks.sn[j] = den > 0.0 ? Hc[j + 1] / den : 0.0;
    Hc[j] = den;
    Hc[j + 1] = 0.0;
    ks.g[j + 1] = -ks.sn[j] * ks.g[j];
    ks.g[j] = ks.cs[j] * ks.g[j];
}

// y = H^{-1} g for the k x k triangle, then coef_i = sign y_i vs_i (thread 0).
FDE_D void solve_triangle(KShared& ks, int k, int m, double sign) {
    for (int i = k - 1; i >= 0; --i) {
        double s = ks.g[i];
        for (int q = i + 1; q < k; ++q) s -= ks.H[i + q * (m + 1)] * ks.y[q];
        ks.y[i] = s / ks.H[i + i * (m + 1)];
    }
    for (int i = 0; i < k; ++i) set_coef(ks, i, sign * ks.y[i] * ks.vs[i]);
}

template <typename W>
FDE_NI bool gmres_right_core(const Team& t, const Inst& I, int lm, const W* rhs, W* sol, const SolveParams& sp,
                             SolveState& st, KShared& ks, const Wk& wk) {
    const long long N = I.N;
    const int m = I.restart;
    GVecs<W> v = gmres_vecs<W>(I);
    long long lo, hi;
    team_range(t, N, lo, hi);
    {
        const W* a[1] = {rhs};
        if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
    }
    const double nb = sqrt(ks.red[0]);
    if (!finite(nb)) {  // NaN or Inf in the right-hand side
        st.relres = st.relres_est = nb;
        st.status = FDE_ENONFINITE;
        return team_sync(t);
    }
    if (!(nb > 0.0)) {  // zero right-hand side: x = 0 is exact
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) sol[i] = W(0);
        st.relres = st.relres_est = 0.0;
        st.status = FDE_OK;
        return team_sync(t);
    }
    st.status = FDE_ENOCONV;
    while (true) {
        // V_0 = rhs - A sol (true residual)
        if (!op_matvec_out<W>(t, I, lm, sol, W(1), v.tt, OutSpec<W>{kOutResid, v.V, rhs}, wk)) return false;
        {
            const W* a[1] = {v.V};
            if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
        }
        const double beta = sqrt(ks.red[0]);
        st.relres = beta / nb;
        if (!finite(beta)) { st.status = FDE_ENONFINITE; break; }
        if (beta <= sp.tol * nb) { st.status = FDE_OK; st.relres_est = beta / nb; break; }
        if (st.iterations >= sp.max_iters) { st.status = FDE_ENOCONV; break; }
        st.cycles++;
        if (threadIdx.x == 0) {
            ks.vs[0] = 1.0 / beta;
            ks.g[0] = beta;
            for (int i = 1; i <= m; ++i) ks.g[i] = 0.0;
        }
        __syncthreads();
        int k = 0;
        int ncoef = 0;             // V_j = w - sum_{q < ncoef} coef_q V_q (j >= 1)
        bool converged = false;
        for (int j = 0; j < m; ++j) {
            Combo<W> u{};
            u.V = v.V;
            u.N = N;
            u.s = W(ks.vs[j]);
            u.base = v.V + (long long)j * N;
            if (j > 0) {
                // V_j = w - sum_q coef_q V_q, streamed once; the transforms then
                // read a plain vector
                trace_mark(t, 24);
                form_basis<W>(t, N, v.w, v.V, kcoef<W>(ks), ncoef, v.V + (long long)j * N);
                if (!team_sync(t)) return false;
                trace_mark(t, 25);
            }
            if (!arnoldi_right<W>(t, I, lm, u, j + 1, v.V, v.z, v.w, v.tt, ks, wk)) return false;
            st.iterations++;
            st.basis_sum += j + 1;
            trace_mark(t, 30);
            // Scalar work is done by thread 0 and broadcast through ks.sc: an
            // FP64 instruction repeated by every warp costs that many times
            // the FP64 pipe.
            if (threadIdx.x == 0) {
                const double ww = ks.red[j + 1];
                const double hh = sum_squares(ks.red, j + 1);
                // ||w - V h|| > eta ||w|| (the Daniel-Gragg-Kaufman-Stewart test):
                // one classical Gram-Schmidt pass is enough.  eta = 1/sqrt(2),
                // except in an FP32 inner solve asked for a loose tolerance: one
                // pass leaves the new vector's orthogonality to the basis at about
                // u ||w|| / ||w - V h||, and while that stays a hundredth of the
                // inner tolerance a second pass buys nothing the outer FP64
                // refinement would see.
                double eta2 = 0.5;
                if (sizeof(W) == 4 && sp.inner) {
                    const double e = 5.96e-8 / (0.01 * sp.tol);
                    eta2 = e * e < 0.5 ? e * e : 0.5;
                }
                const bool once = ww - hh > eta2 * ww;
                ks.sc[0] = once ? 0.0 : 1.0;
                ks.sc[1] = ww - hh;
                if (once) {
                    // V_{j+1} = w - sum h_q vs_q V_q (formed by the next step)
                    for (int q = 0; q <= j; ++q) {
                        ks.H[q + j * (m + 1)] = ks.red[q];
                        set_coef(ks, q, ks.red[q] * ks.vs[q]);
                    }
                }
            }
            __syncthreads();
            if (ks.sc[0] != 0.0) {
                st.reorth++;
                // reorthogonalise: w <- w - V h, then h2 = V^T w (V_j was stored
                // by this step's first phase; the team barrier of the reduction
                // made it visible)
                if (threadIdx.x <= j) {
                    set_coef(ks, threadIdx.x, ks.red[threadIdx.x] * ks.vs[threadIdx.x]);
                    ks.y[threadIdx.x] = ks.red[threadIdx.x];
                }
                __syncthreads();
                form_basis<W>(t, N, v.w, v.V, kcoef<W>(ks), j + 1, v.w);
                __syncthreads();
                trace_mark(t, 32);
                if (!dots_basis<W>(t, N, v.w, v.V, ks.vs, j + 1, true, ks)) return false;
                trace_mark(t, 31);
                if (threadIdx.x == 0) ks.sc[1] = ks.red[j + 1] - sum_squares(ks.red, j + 1);
                if (threadIdx.x <= j) {
                    ks.H[threadIdx.x + j * (m + 1)] = ks.y[threadIdx.x] + ks.red[threadIdx.x];
                    set_coef(ks, threadIdx.x, ks.red[threadIdx.x] * ks.vs[threadIdx.x]);
                }
                __syncthreads();
            }
            ncoef = j + 1;
            if (threadIdx.x == 0) {
                const double hn2 = ks.sc[1];
                const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
                ks.H[(j + 1) + j * (m + 1)] = hn;
                givens_column(ks, j, m);
                ks.vs[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
                const double est = fabs(ks.g[j + 1]);
                const double diag = ks.H[j + j * (m + 1)];
                double flag = 0.0;
                if (!finite(est) || !finite(hn)) flag = 1.0;
                else if (est <= sp.tol * nb || !(hn > 1e-14 * diag)) flag = 2.0;   // converged or breakdown
                ks.sc[2] = est / nb;
                ks.sc[3] = flag;
            }
            __syncthreads();
            k = j + 1;
            st.relres_est = ks.sc[2];
            const double flag = ks.sc[3];
            __syncthreads();   // ks.sc is rewritten by the next step's thread 0
            if (flag == 1.0) { st.status = FDE_ENONFINITE; break; }
            if (flag == 2.0) { converged = true; break; }
            if (st.iterations >= sp.max_iters) break;
        }
        if (st.status == FDE_ENONFINITE) break;
        // sol += P^{-1} (sum_i y_i vs_i V_i), the combination formed on the fly
        if (threadIdx.x == 0) solve_triangle(ks, k, m, -1.0);
        __syncthreads();
        Combo<W> upd{};
        upd.V = v.V;
        upd.c = kcoef<W>(ks);
        upd.cnt = k;
        upd.N = N;
        upd.s = W(1);
        if (!op_tau_combo<W>(t, I, lm, upd, v.z, OutSpec<W>{kOutAdd, sol, nullptr}, wk)) return false;
        if (sp.inner && (converged || st.iterations >= sp.max_iters)) {
            // An inner solve trusts its estimate: below the working precision's
            // floor a recomputed residual says nothing the outer FP64 residual won't.
            st.status = converged ? FDE_OK : FDE_ENOCONV;
            break;
        }
        st.restarts++;
    }
    return team_sync(t);
}

template <typename W>
FDE_NI bool gmres_left_core(const Team& t, const Inst& I, int lm, const W* rhs, W* sol, const SolveParams& sp,
                            SolveState& st, KShared& ks, const Wk& wk) {
    const long long N = I.N;
    const int m = I.restart;
    GVecs<W> v = gmres_vecs<W>(I);
    long long lo, hi;
    team_range(t, N, lo, hi);
    {
        const W* a[1] = {rhs};
        if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
    }
    const double nb = sqrt(ks.red[0]);
    if (!finite(nb)) {  // NaN or Inf in the right-hand side
        st.relres = st.relres_est = nb;
        st.status = FDE_ENONFINITE;
        return team_sync(t);
    }
    if (!(nb > 0.0)) {  // zero right-hand side: x = 0 is exact
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) sol[i] = W(0);
        st.relres = st.relres_est = 0.0;
        st.status = FDE_OK;
        return team_sync(t);
    }
    double ref = nb;       // ||P^-1 r_0||
    bool first = true;
    st.status = FDE_ENOCONV;
    while (true) {
        if (!op_matvec_out<W>(t, I, lm, sol, W(1), v.tt, OutSpec<W>{kOutResid, v.z, rhs}, wk)) return false;
        {
            const W* a[1] = {v.z};
            if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
        }
        st.relres = sqrt(ks.red[0]) / nb;
        if (!op_tau<W>(t, I, lm, v.z, W(1), v.V, wk)) return false;
        {
            const W* a[1] = {v.V};
            if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
        }
        const double beta = sqrt(ks.red[0]);
        if (first) ref = beta;
        first = false;
        if (!finite(beta)) { st.status = FDE_ENONFINITE; break; }
        if (beta <= sp.tol * ref || beta == 0.0) { st.status = FDE_OK; st.relres_est = beta / ref; break; }
        if (st.iterations >= sp.max_iters) { st.status = FDE_ENOCONV; break; }
        st.cycles++;
        if (threadIdx.x == 0) {
            ks.vs[0] = 1.0 / beta;
            ks.g[0] = beta;
            for (int i = 1; i <= m; ++i) ks.g[i] = 0.0;
        }
        __syncthreads();
        int k = 0;
        bool converged = false;
        for (int j = 0; j < m; ++j) {
            if (!op_matvec<W>(t, I, lm, v.V + (long long)j * N, W(ks.vs[j]), v.z, v.tt, wk)) return false;
            if (!op_tau<W>(t, I, lm, v.z, W(1), v.w, wk)) return false;
            st.iterations++;
            st.basis_sum += j + 1;
            st.reorth++;               // the left variant always takes two passes
            if (!dots_basis<W>(t, N, v.w, v.V, ks.vs, j + 1, false, ks)) return false;
            if (threadIdx.x <= j) {
                ks.y[threadIdx.x] = ks.red[threadIdx.x];
                set_coef(ks, threadIdx.x, ks.red[threadIdx.x] * ks.vs[threadIdx.x]);
            }
            __syncthreads();
            const W* kc = kcoef<W>(ks);
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                W acc = ldw(v.w + i);
                for (int q = 0; q <= j; ++q) acc -= kc[q] * ldw(v.V + (long long)q * N + i);
                v.w[i] = acc;
            }
            __syncthreads();
            if (!dots_basis<W>(t, N, v.w, v.V, ks.vs, j + 1, true, ks)) return false;
            double s2 = 0.0;
            for (int q = 0; q <= j; ++q) s2 += ks.red[q] * ks.red[q];
            const double hn2 = ks.red[j + 1] - s2;
            const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
            __syncthreads();
            if (threadIdx.x <= j) set_coef(ks, threadIdx.x, ks.red[threadIdx.x] * ks.vs[threadIdx.x]);
            __syncthreads();
            W* vn = v.V + (long long)(j + 1) * N;
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                W acc = ldw(v.w + i);
                for (int q = 0; q <= j; ++q) acc -= kc[q] * ldw(v.V + (long long)q * N + i);
                vn[i] = acc;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int q = 0; q <= j; ++q) ks.H[q + j * (m + 1)] = ks.y[q] + ks.red[q];
                ks.H[(j + 1) + j * (m + 1)] = hn;
                givens_column(ks, j, m);
                ks.vs[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
            }
            if (!team_sync(t)) return false;
            const double est = fabs(ks.g[j + 1]);
            const double diag = ks.H[j + j * (m + 1)];
            k = j + 1;
            st.relres_est = est / ref;
            if (!finite(est) || !finite(hn)) { st.status = FDE_ENONFINITE; break; }
            const bool breakdown = !(hn > 1e-14 * diag);
            if (est <= sp.tol * ref || breakdown) { converged = true; break; }
            if (st.iterations >= sp.max_iters) break;
        }
        if (st.status == FDE_ENONFINITE) break;
        if (threadIdx.x == 0) solve_triangle(ks, k, m, 1.0);
        __syncthreads();
        {
            const W* kc = kcoef<W>(ks);
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                W acc = sol[i];
                for (int q = 0; q < k; ++q) acc += kc[q] * ldw(v.V + (long long)q * N + i);
                sol[i] = acc;
            }
        }
        if (!team_sync(t)) return false;
        if (sp.inner && (converged || st.iterations >= sp.max_iters)) {
            st.status = converged ? FDE_OK : FDE_ENOCONV;
            break;
        }
        st.restarts++;
    }
    return team_sync(t);
}

// ---------------------------------------------------------------------------
// PCG
// ---------------------------------------------------------------------------

template <typename W>
FDE_NI bool pcg_core(const Team& t, const Inst& I, int lm, const W* rhs, W* sol, const SolveParams& sp,
                     SolveState& st, KShared& ks, const Wk& wk) {
    const long long N = I.N;
    W* base = reinterpret_cast<W*>(I.wvec);
    W* r = base;
    W* z = base + N;
    W* p = base + 2 * N;
    W* q = base + 3 * N;
    W* tt = base + 4 * N;
    long long lo, hi;
    team_range(t, N, lo, hi);
    {
        const W* a[1] = {rhs};
        if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
    }
    const double nb = sqrt(ks.red[0]);
    if (!finite(nb)) {  // NaN or Inf in the right-hand side
        st.relres = st.relres_est = nb;
        st.status = FDE_ENONFINITE;
        return team_sync(t);
    }
    if (!(nb > 0.0)) {  // zero right-hand side: x = 0 is exact
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) sol[i] = W(0);
        st.relres = st.relres_est = 0.0;
        st.status = FDE_OK;
        return team_sync(t);
    }
    // A pass starts from the true residual r = rhs - A sol.  It ends when the
    // recurrence's residual meets the tolerance; the next pass's true residual
    // then decides.  Where rounding has moved the recurrence away from the true
    // residual (tight tolerances), PCG restarts from the true one, at most
    // kPcgPasses - 1 times, and reports FDE_ENOCONV if that still falls short.
    constexpr int kPcgPasses = 3;
    st.status = FDE_ENOCONV;
    for (int pass = 0;; ++pass) {
        if (!op_matvec_out<W>(t, I, lm, sol, W(1), tt, OutSpec<W>{kOutResid, r, rhs}, wk)) return false;
        {
            const W* a[1] = {r};
            if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
        }
        double rr = ks.red[0];
        st.relres = sqrt(rr) / nb;
        if (pass == 0) st.relres_est = st.relres;
        if (st.status == FDE_ENONFINITE || st.status == FDE_EBREAKDOWN) break;
        if (!finite(rr)) { st.status = FDE_ENONFINITE; break; }
        if (sqrt(rr) <= sp.tol * nb) { st.status = FDE_OK; break; }
        st.status = FDE_ENOCONV;
        if (pass >= kPcgPasses - 1 || st.iterations >= sp.max_iters) break;
        st.cycles++;
        if (!op_tau<W>(t, I, lm, r, W(1), z, wk)) return false;
        {
            const W* a[1] = {r};
            const W* b[1] = {z};
            if (!dots_pairs<W, 1>(t, N, a, b, ks)) return false;
        }
        double rz = ks.red[0];
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) p[i] = ldw(z + i);
        if (!team_sync(t)) return false;
        bool recurrence_met = false;
        while (st.iterations < sp.max_iters) {
            if (!op_matvec<W>(t, I, lm, p, W(1), q, tt, wk)) return false;
            st.iterations++;
            {
                const W* a[1] = {p};
                const W* b[1] = {q};
                if (!dots_pairs<W, 1>(t, N, a, b, ks)) return false;
            }
            // scalars by thread 0, broadcast through ks.sc (see gmres_right_core)
            if (threadIdx.x == 0) {
                const double pq = ks.red[0];
                ks.sc[0] = !finite(pq) ? 1.0 : (!(pq > 0.0) ? 2.0 : 0.0);
                ks.sc[1] = rz / pq;
            }
            __syncthreads();
            if (ks.sc[0] == 1.0) { st.status = FDE_ENONFINITE; break; }
            if (ks.sc[0] == 2.0) { st.status = FDE_EBREAKDOWN; break; }
            const W alw = W(ks.sc[1]);
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                sol[i] = sol[i] + alw * ldw(p + i);
                r[i] = ldw(r + i) - alw * ldw(q + i);
            }
            __syncthreads();
            {
                const W* a[1] = {r};
                if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
            }
            if (threadIdx.x == 0) {
                const double rrn = ks.red[0];
                const double nr = sqrt(rrn);
                ks.sc[2] = nr / nb;
                ks.sc[3] = !finite(rrn) ? 1.0 : (nr <= sp.tol * nb ? 2.0 : 0.0);
            }
            __syncthreads();
            st.relres_est = ks.sc[2];
            if (ks.sc[3] == 1.0) { st.status = FDE_ENONFINITE; break; }
            if (ks.sc[3] == 2.0) { recurrence_met = true; break; }
            if (!op_tau<W>(t, I, lm, r, W(1), z, wk)) return false;
            {
                const W* a[1] = {r};
                const W* b[1] = {z};
                if (!dots_pairs<W, 1>(t, N, a, b, ks)) return false;
            }
            if (threadIdx.x == 0) {
                const double rz_new = ks.red[0];
                ks.sc[4] = rz_new / rz;
                rz = rz_new;
            }
            __syncthreads();
            const W bew = W(ks.sc[4]);
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) p[i] = ldw(z + i) + bew * ldw(p + i);
            if (!team_sync(t)) return false;
        }
        if (sp.inner) {
            // an inner solve of the refinement trusts its recurrence (the outer
            // loop recomputes the residual in FP64)
            if (recurrence_met) st.status = FDE_OK;
            st.relres = st.relres_est;
            return team_sync(t);
        }
    }
    return team_sync(t);
}

template <typename W>
FDE_D bool krylov_core(const Team& t, const Inst& I, int lm, const W* rhs, W* sol, const SolveParams& sp,
                       SolveState& st, KShared& ks, const Wk& wk) {
    if (I.method == FDE_PCG) return pcg_core<W>(t, I, lm, rhs, sol, sp, st, ks, wk);
    if (sp.side == FDE_SIDE_LEFT) return gmres_left_core<W>(t, I, lm, rhs, sol, sp, st, ks, wk);
    return gmres_right_core<W>(t, I, lm, rhs, sol, sp, st, ks, wk);
}

}  // namespace fde
