// Device-resident Krylov drivers: PCG and restarted GMRES(m) (right or left
// preconditioned, classical Gram-Schmidt with one reorthogonalisation), and
// the FP32-inner / FP64-outer iterative refinement around them.  Every CTA of
// a team runs the same scalar recurrences on the same deterministic
// reductions, so all CTAs take identical decisions without extra barriers.
// Inner products, norms, the Hessenberg matrix and the Givens rotations are
// FP64 whatever the vector precision.
#pragma once

#include "ops.cuh"

namespace fde {

struct SolveParams {
    double tol;            // relative to ||rhs||
    int max_iters;         // cap on products with M
    int side;              // FDE_SIDE_RIGHT / FDE_SIDE_LEFT
    int inner;             // inner solve of a refinement: stop on the Krylov estimate, no FP32 true residual
};

struct SolveState {
    int iterations;
    int restarts;
    int status;
    double relres_est;
    double relres;         // true residual of the last check, relative to ||rhs||
};

// Shared-memory scalars of one CTA (identical in every CTA of a team).
struct KShared {
    double* H;             // (m+1) x m, column-major H[i + j (m+1)]
    double* cs;
    double* sn;
    double* g;
    double* y;
    double* vs;            // 1/||v_i|| of the stored (unnormalised) basis vectors
    double* red;           // reduction results, kMaxDots + 8
    double* scratch;       // 8 * 32 for block_sum
    double* coef;          // per-basis coefficients for fused updates
};

FDE_HD size_t kshared_bytes(int m) {
    size_t d = (size_t)(m + 1) * m + 3 * (size_t)m + 2 * (size_t)(m + 2) + (kMaxDots + 8) + 8 * 32 + (m + 2);
    return ((d * sizeof(double)) + 255) & ~(size_t)255;
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
    k.scratch = p; p += 8 * 32;
    k.coef = p;
    return k;
}

FDE_D bool finite(double v) { return isfinite(v); }

// ---------------------------------------------------------------------------
// Reductions over N-vectors
// ---------------------------------------------------------------------------

// out[i] = <a, vs_i V_i> for i < cnt (V_i at V + i N); with `norm`, also
// out[cnt] = <a, a>.  Team-wide totals in every CTA.
template <typename W>
FDE_D bool dots_basis(const Team& t, long long N, const W* a, const W* V, const double* vs, int cnt, bool norm,
                      KShared& ks) {
    long long lo, hi;
    team_range(t, N, lo, hi);
    const int tot = cnt + (norm ? 1 : 0);
    for (int c0 = 0; c0 < tot; c0 += 8) {
        double acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.0;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double ai = (double)ldw(a + i);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int kk = c0 + k;
                if (kk < cnt) acc[k] += ai * (double)ldw(V + (long long)kk * N + i);
                else if (kk == cnt && norm) acc[k] += ai * ai;
            }
        }
        block_sum<8>(acc, ks.red + c0, ks.scratch);
    }
    if (threadIdx.x < cnt) ks.red[threadIdx.x] *= vs[threadIdx.x];
    __syncthreads();
    return team_allreduce(t, ks.red, tot);
}

// out[k] = <a_k, b_k> for up to 4 pairs (any pointer may repeat).
template <typename W, int K>
FDE_D bool dots_pairs(const Team& t, long long N, const W* const (&a)[K], const W* const (&b)[K], KShared& ks) {
    long long lo, hi;
    team_range(t, N, lo, hi);
    double acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += (double)ldw(a[k] + i) * (double)ldw(b[k] + i);
    }
    block_sum<8>(acc, ks.red, ks.scratch);
    return team_allreduce(t, ks.red, K);
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

template <typename W>
FDE_NI bool gmres_core(const Team& t, const Inst& I, int lm, const W* rhs, W* sol, const SolveParams& sp,
                      SolveState& st, KShared& ks, unsigned char* work, int bytes) {
    const long long N = I.N;
    const int m = I.restart;
    const bool left = sp.side == FDE_SIDE_LEFT;
    GVecs<W> v = gmres_vecs<W>(I);
    long long lo, hi;
    team_range(t, N, lo, hi);

    // ||rhs||
    {
        const W* a[1] = {rhs};
        if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
    }
    const double nb = sqrt(ks.red[0]);
    if (!(nb > 0.0)) {  // zero right-hand side: x = 0 is exact
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) sol[i] = W(0);
        st.relres = 0.0;
        st.relres_est = 0.0;
        st.status = FDE_OK;
        return team_sync(t);
    }
    double ref = nb;       // left: ||P^-1 r_0||
    bool first = true;
    st.status = FDE_ENOCONV;
    while (true) {
        // r = rhs - A sol into V_0 (left: P^-1 of it)
        if (!op_matvec<W>(t, I, lm, sol, W(1), v.w, v.tt, work, bytes)) return false;
        W* rdst = left ? v.z : v.V;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) rdst[i] = ldw(rhs + i) - ldw(v.w + i);
        if (!team_sync(t)) return false;
        double beta, true_rel;
        {
            const W* a[1] = {rdst};
            if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
            true_rel = sqrt(ks.red[0]) / nb;
        }
        if (left) {
            if (!op_tau<W>(t, I, lm, v.z, W(1), v.V, work, bytes)) return false;
            const W* a[1] = {v.V};
            if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
            beta = sqrt(ks.red[0]);
            if (first) ref = beta;
        } else {
            beta = true_rel * nb;
        }
        first = false;
        st.relres = true_rel;
        if (!finite(beta)) { st.status = FDE_ENONFINITE; break; }
        if (beta <= sp.tol * ref || (left && beta == 0.0)) { st.status = FDE_OK; st.relres_est = beta / ref; break; }
        if (st.iterations >= sp.max_iters) { st.status = FDE_ENOCONV; break; }
        if (threadIdx.x == 0) {
            ks.vs[0] = 1.0 / beta;
            ks.g[0] = beta;
            for (int i = 1; i <= m; ++i) ks.g[i] = 0.0;
        }
        __syncthreads();
        int k = 0;
        bool cycle_converged = false;
        for (int j = 0; j < m; ++j) {
            const W sj = W(ks.vs[j]);
            const W* vj = v.V + (long long)j * N;
            if (left) {
                if (!op_matvec<W>(t, I, lm, vj, sj, v.z, v.tt, work, bytes)) return false;
                if (!op_tau<W>(t, I, lm, v.z, W(1), v.w, work, bytes)) return false;
            } else {
                if (!op_tau<W>(t, I, lm, vj, sj, v.z, work, bytes)) return false;
                if (!op_matvec<W>(t, I, lm, v.z, W(1), v.w, v.tt, work, bytes)) return false;
            }
            st.iterations++;
            // pass 1: h = V^T w
            if (!dots_basis<W>(t, N, v.w, v.V, ks.vs, j + 1, false, ks)) return false;
            if (threadIdx.x <= j) ks.coef[threadIdx.x] = ks.red[threadIdx.x];
            __syncthreads();
            // w <- w - V h; pass 2: h2 = V^T w, ||w||^2
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                double acc = (double)ldw(v.w + i);
                for (int q = 0; q <= j; ++q) acc -= ks.coef[q] * ks.vs[q] * (double)ldw(v.V + (long long)q * N + i);
                v.w[i] = W(acc);
            }
            __syncthreads();
            if (!dots_basis<W>(t, N, v.w, v.V, ks.vs, j + 1, true, ks)) return false;
            double hn2 = ks.red[j + 1];
            if (threadIdx.x == 0) {
                double s2 = 0.0;
                for (int q = 0; q <= j; ++q) {
                    ks.H[q + j * (m + 1)] = ks.coef[q] + ks.red[q];
                    s2 += ks.red[q] * ks.red[q];
                }
                ks.y[0] = hn2 - s2;       // ||w - V h2||^2
            }
            __syncthreads();
            hn2 = ks.y[0];
            const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
            // V_{j+1} = w - V h2 (unnormalised), scale 1/hn
            W* vn = v.V + (long long)(j + 1) * N;
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                double acc = (double)ldw(v.w + i);
                for (int q = 0; q <= j; ++q) acc -= ks.red[q] * ks.vs[q] * (double)ldw(v.V + (long long)q * N + i);
                vn[i] = W(acc);
            }
            double hnorm_ref = 0.0;
            if (threadIdx.x == 0) {
                double* Hc = ks.H + j * (m + 1);
                Hc[j + 1] = hn;
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
                ks.vs[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
                ks.y[1] = den;
            }
            if (!team_sync(t)) return false;
            hnorm_ref = ks.y[1];
            const double est = fabs(ks.g[j + 1]);
            k = j + 1;
            st.relres_est = est / ref;
            if (!finite(est) || !finite(hn)) { st.status = FDE_ENONFINITE; break; }
            const bool breakdown = !(hn > 1e-14 * hnorm_ref);
            if (est <= sp.tol * ref || breakdown) { cycle_converged = true; break; }
            if (st.iterations >= sp.max_iters) break;
        }
        if (st.status == FDE_ENONFINITE) break;
        // y = H^{-1} g (k x k upper triangular), u = sum y_i vs_i V_i
        if (threadIdx.x == 0) {
            for (int i = k - 1; i >= 0; --i) {
                double s = ks.g[i];
                for (int q = i + 1; q < k; ++q) s -= ks.H[i + q * (m + 1)] * ks.y[q];
                ks.y[i] = s / ks.H[i + i * (m + 1)];
            }
            for (int i = 0; i < k; ++i) ks.coef[i] = ks.y[i] * ks.vs[i];
        }
        __syncthreads();
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            double acc = 0.0;
            for (int q = 0; q < k; ++q) acc += ks.coef[q] * (double)ldw(v.V + (long long)q * N + i);
            v.tt[i] = W(acc);
        }
        if (!team_sync(t)) return false;
        if (!left) {
            if (!op_tau<W>(t, I, lm, v.tt, W(1), v.z, work, bytes)) return false;
        }
        const W* upd = left ? v.tt : v.z;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) sol[i] = sol[i] + ldw(upd + i);
        if (!team_sync(t)) return false;
        // An inner solve trusts its estimate: below the working precision's
        // floor a recomputed residual says nothing the outer FP64 residual won't.
        if (sp.inner && (cycle_converged || st.iterations >= sp.max_iters)) {
            st.status = cycle_converged ? FDE_OK : FDE_ENOCONV;
            break;
        }
        st.restarts++;
        // loop: the true residual at the top decides
    }
    return team_sync(t);
}

// ---------------------------------------------------------------------------
// PCG
// ---------------------------------------------------------------------------

template <typename W>
FDE_NI bool pcg_core(const Team& t, const Inst& I, int lm, const W* rhs, W* sol, const SolveParams& sp,
                    SolveState& st, KShared& ks, unsigned char* work, int bytes) {
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
    if (!(nb > 0.0)) {
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) sol[i] = W(0);
        st.relres = st.relres_est = 0.0;
        st.status = FDE_OK;
        return team_sync(t);
    }
    if (!op_matvec<W>(t, I, lm, sol, W(1), q, tt, work, bytes)) return false;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) r[i] = ldw(rhs + i) - ldw(q + i);
    if (!team_sync(t)) return false;
    {
        const W* a[1] = {r};
        if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
    }
    double rr = ks.red[0];
    st.relres = st.relres_est = sqrt(rr) / nb;
    st.status = FDE_ENOCONV;
    if (sqrt(rr) <= sp.tol * nb) { st.status = FDE_OK; return team_sync(t); }
    if (!op_tau<W>(t, I, lm, r, W(1), z, work, bytes)) return false;
    {
        const W* a[1] = {r};
        const W* b[1] = {z};
        if (!dots_pairs<W, 1>(t, N, a, b, ks)) return false;
    }
    double rz = ks.red[0];
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) p[i] = ldw(z + i);
    if (!team_sync(t)) return false;
    while (st.iterations < sp.max_iters) {
        if (!op_matvec<W>(t, I, lm, p, W(1), q, tt, work, bytes)) return false;
        st.iterations++;
        {
            const W* a[1] = {p};
            const W* b[1] = {q};
            if (!dots_pairs<W, 1>(t, N, a, b, ks)) return false;
        }
        const double pq = ks.red[0];
        if (!finite(pq)) { st.status = FDE_ENONFINITE; break; }
        if (!(pq > 0.0)) { st.status = FDE_EBREAKDOWN; break; }
        const double al = rz / pq;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            sol[i] = W((double)sol[i] + al * (double)ldw(p + i));
            r[i] = W((double)ldw(r + i) - al * (double)ldw(q + i));
        }
        if (!team_sync(t)) return false;
        {
            const W* a[1] = {r};
            if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
        }
        rr = ks.red[0];
        st.relres_est = sqrt(rr) / nb;
        if (!finite(rr)) { st.status = FDE_ENONFINITE; break; }
        if (sqrt(rr) <= sp.tol * nb) { st.status = FDE_OK; break; }
        if (!op_tau<W>(t, I, lm, r, W(1), z, work, bytes)) return false;
        {
            const W* a[1] = {r};
            const W* b[1] = {z};
            if (!dots_pairs<W, 1>(t, N, a, b, ks)) return false;
        }
        const double rz_new = ks.red[0];
        const double be = rz_new / rz;
        rz = rz_new;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) p[i] = W((double)ldw(z + i) + be * (double)ldw(p + i));
        if (!team_sync(t)) return false;
    }
    if (sp.inner) {
        st.relres = st.relres_est;
        return team_sync(t);
    }
    // true residual of the final iterate
    if (!op_matvec<W>(t, I, lm, sol, W(1), q, tt, work, bytes)) return false;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) r[i] = ldw(rhs + i) - ldw(q + i);
    if (!team_sync(t)) return false;
    {
        const W* a[1] = {r};
        if (!dots_pairs<W, 1>(t, N, a, a, ks)) return false;
    }
    st.relres = sqrt(ks.red[0]) / nb;
    return team_sync(t);
}

template <typename W>
FDE_D bool krylov_core(const Team& t, const Inst& I, int lm, const W* rhs, W* sol, const SolveParams& sp,
                       SolveState& st, KShared& ks, unsigned char* work, int bytes) {
    if (I.method == FDE_PCG) return pcg_core<W>(t, I, lm, rhs, sol, sp, st, ks, work, bytes);
    return gmres_core<W>(t, I, lm, rhs, sol, sp, st, ks, work, bytes);
}

}  // namespace fde
