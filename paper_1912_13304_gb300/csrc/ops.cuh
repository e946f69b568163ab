// The two operators of one Krylov iteration, for every data layout:
//   op_matvec: y = M (s x)      (Sec. 1.2 / 1.4, Toeplitz by circulant embedding)
//   op_tau:    z = P^{-1} (s r) (Sec. 3.1 / 3.2, DST-I / symbol / DST-I)
// Layouts: a 1D line held whole by one CTA; a 1D line split across the CTAs
// of a team (Np = P1 * P2, column / row / column phases through an L2-resident
// intermediate); a 2D plane (row lines along x, column lines along y).
// Every operator ends with a team barrier, so its output is complete on return.
#pragma once

#include "lines.cuh"

namespace fde {

template <typename W> struct Ept { static constexpr int v = sizeof(W) == 4 ? 32 : 16; };

template <typename W>
FDE_D W coef(const W* arr, double cst, long long i) {
    return arr ? __ldg(arr + i) : W(cst);
}

// Lines of Np complex values that fit the register staging of fft_inplace and
// `bytes` of shared memory, with `nbuf` buffers per line.
template <typename W>
FDE_HD int max_lines(int Np, int nbuf, int bytes) {
    const int by_regs = (Ept<W>::v * kThreads) / (Np * nbuf);
    const int by_smem = bytes / (int)(Np * nbuf * sizeof(cx<W>));
    int b = by_regs < by_smem ? by_regs : by_smem;
    return b;
}

FDE_D int pow2_floor(int v) { int p = 1; while (p * 2 <= v) p *= 2; return p; }

// ---------------------------------------------------------------------------
// Multipliers
// ---------------------------------------------------------------------------

template <typename W>
FDE_D Mult<W> mult_matvec(const AxisData& A, bool sym) {
    Mult<W> mu{};
    mu.kind = sym ? kMulSym : kMulLam2;
    mu.lam = Prec<W>::lam(A);
    mu.n = A.n;
    mu.Np = A.Np;
    return mu;
}

template <typename W>
FDE_D Mult<W> mult_tau1(const AxisData& A) {
    Mult<W> mu{};
    mu.kind = kMulTau1;
    mu.phi = Prec<W>::phi(A);
    mu.n = A.n;
    mu.Np = A.Np;
    return mu;
}

template <typename W>
FDE_D Mult<W> mult_tau2(const Inst& I) {
    Mult<W> mu{};
    mu.kind = kMulTau2;
    mu.phi = Prec<W>::phi(I.ax[1]);
    mu.a1 = Prec<W>::phi(I.ax[0]);
    mu.scale2d = W(I.phi_scale2d);
    mu.n = I.ax[1].n;
    mu.Np = I.ax[1].Np;
    return mu;
}

// ---------------------------------------------------------------------------
// 1D, whole line in one CTA
// ---------------------------------------------------------------------------

template <typename W>
FDE_NI void cta_matvec_1d(const Inst& I, const W* x, W s, W* y, unsigned char* work) {
    const AxisData& A = I.ax[0];
    const int n = A.n, Np = A.Np;
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    cx<W>* buf2 = buf + Np;
    const bool sym = I.symx;
    const RealIn<W> in{x, 1, s, nullptr};
    cta_pack<W, kExtZero, false>(buf, 1, n, Np, [&](int) { return in; });
    fft_inplace<W, Ept<W>::v, false>(buf, A.logNp, 1, Np, Prec<W>::tw(I), I.logTW);
    const Mult<W> mu = mult_matvec<W>(A, sym);
    cta_spectral<W>(buf, buf2, 1, Np, A.logNp, Prec<W>::tw(I), I.logTW, mu, [](int) { return 0; });
    fft_inplace<W, Ept<W>::v, true>(buf, A.logNp, sym ? 1 : 2, Np, Prec<W>::tw(I), I.logTW);
    const W c0s = W(I.c0) * s;
    const W* dp = Prec<W>::dp(I);
    const W* dm = Prec<W>::dm(I);
    if (sym) {
        cta_unpack<W, false, false>(buf, buf2, 1, n, Np, [&](int, int p, W va, W) {
            y[p] = c0s * ldw(x + p) + coef(dp, I.dpc, p) * va;
        });
    } else {
        cta_unpack<W, false, true>(buf, buf2, 1, n, Np, [&](int, int p, W va, W vb) {
            y[p] = c0s * ldw(x + p) + coef(dp, I.dpc, p) * va + coef(dm, I.dmc, p) * vb;
        });
    }
    __syncthreads();
}

template <typename W>
FDE_NI void cta_tau_1d(const Inst& I, const W* r, W s, W* z, unsigned char* work) {
    const AxisData& A = I.ax[0];
    const int n = A.n, Np = A.Np;
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    const W* dinv = Prec<W>::dinv(I);
    const bool pre = I.has_D && I.order == FDE_ORDER_D_TAU;
    const bool post = I.has_D && I.order == FDE_ORDER_TAU_D;
    const RealIn<W> in{r, 1, s, pre ? dinv : nullptr};
    cta_pack<W, kExtOdd, false>(buf, 1, n, Np, [&](int) { return in; });
    fft_inplace<W, Ept<W>::v, false>(buf, A.logNp, 1, Np, Prec<W>::tw(I), I.logTW);
    const Mult<W> mu = mult_tau1<W>(A);
    cta_spectral<W>(buf, nullptr, 1, Np, A.logNp, Prec<W>::tw(I), I.logTW, mu, [](int) { return 0; });
    fft_inplace<W, Ept<W>::v, true>(buf, A.logNp, 1, Np, Prec<W>::tw(I), I.logTW);
    cta_unpack<W, false, false>(buf, nullptr, 1, n, Np, [&](int, int p, W va, W) {
        z[p] = post ? va * __ldg(dinv + p) : va;
    });
    __syncthreads();
}

// ---------------------------------------------------------------------------
// 1D, line split across a team: Np = P1 * P2, m = P2 m1 + m2, j = j1 + P1 j2.
// ---------------------------------------------------------------------------

template <typename W>
FDE_D int split_cols_per_unit(const AxisData& A, int team_size, int nbuf, int bytes) {
    int cap = max_lines<W>(A.P1, nbuf, bytes);
    int want = A.P2 / team_size;
    int cc = 1;
    while (cc < want) cc *= 2;          // units <= team size when possible
    if (cc > cap) cc = pow2_floor(cap);
    if (cc > A.P2) cc = A.P2;
    if (cc < 1) cc = 1;
    return cc;
}

// Column phase of the forward transform: pack, P1-point FFTs, twiddle,
// store Y[j1][m2].
template <typename W, int EXT>
FDE_NI void split_fwd_cols(const Team& t, const Inst& I, const RealIn<W>& in, cx<W>* Y, unsigned char* work,
                          int cc) {
    const AxisData& A = I.ax[0];
    const int n = A.n, Np = A.Np, P1 = A.P1, P2 = A.P2;
    const cx<W>* tw = Prec<W>::tw(I);
    const int tsh = I.logTW - A.logNp;
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    const int units = P2 / cc;
    for (int u = t.rank; u < units; u += t.size) {
        const int m2b = u * cc;
        for (int idx = threadIdx.x; idx < cc * P1; idx += blockDim.x) {
            const int c = idx % cc, m1 = idx / cc;
            buf[c * P1 + m1] = pack_elem<W, EXT>(in, P2 * m1 + m2b + c, n, Np);
        }
        __syncthreads();
        fft_inplace<W, Ept<W>::v, false>(buf, A.logP1, cc, P1, tw, I.logTW);
        for (int idx = threadIdx.x; idx < cc * P1; idx += blockDim.x) {
            const int c = idx % cc, j1 = idx / cc;
            const int m2 = m2b + c;
            Y[(long long)j1 * P2 + m2] = buf[c * P1 + j1] * tw[(j1 * m2) << tsh];
        }
        __syncthreads();
    }
}

// Row phase: P2-point FFTs of rows {j1, P1-j1}, the spectral step on the
// pairs (j, Np-j), inverse P2-point FFTs, inverse twiddle; results back to Y
// (and Y2 for the second multiplier).
template <typename W>
FDE_NI void split_rows(const Team& t, const Inst& I, const Mult<W>& mu, cx<W>* Y, cx<W>* Y2,
                      unsigned char* work) {
    const AxisData& A = I.ax[0];
    const int P1 = A.P1, P2 = A.P2;
    const cx<W>* tw = Prec<W>::tw(I);
    const int wsh = I.logTW - (A.logNp + 1);
    const int tsh = I.logTW - A.logNp;
    const bool two = mu.kind == kMulLam2;
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    const int units = P1 / 2 + 1;
    for (int u = t.rank; u < units; u += t.size) {
        const int nrows = u < 2 ? 1 : 2;
        int rows[2];
        rows[0] = u == 0 ? 0 : (u == 1 ? P1 / 2 : u - 1);
        rows[1] = P1 - rows[0];
        cx<W>* buf2 = buf + nrows * P2;
        for (int idx = threadIdx.x; idx < nrows * P2; idx += blockDim.x) {
            const int sl = idx / P2, j2 = idx - sl * P2;
            buf[idx] = ldw(Y + (long long)rows[sl] * P2 + j2);
        }
        __syncthreads();
        fft_inplace<W, Ept<W>::v, false>(buf, A.logP2, nrows, P2, tw, I.logTW);
        const int npairs = u == 0 ? P2 / 2 + 1 : (u == 1 ? P2 / 2 : P2);
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            int sj, j2, sm, j2m;
            if (u == 0) { sj = 0; j2 = q; sm = 0; j2m = (P2 - q) & (P2 - 1); }
            else if (u == 1) { sj = 0; j2 = q; sm = 0; j2m = P2 - 1 - q; }
            else { sj = 0; j2 = q; sm = 1; j2m = P2 - 1 - q; }
            const int j = rows[sj] + P1 * j2;              // frequency of the first element
            const cx<W> wj = tw[j << wsh];
            cx<W> a, b, al, be, al2, be2;
            unpack_pair(buf[sj * P2 + j2], buf[sm * P2 + j2m], wj, a, b);
            mu.apply(j, 0, a, b, al, be, al2, be2);
            cx<W> Qj, Qm;
            repack_pair(al, be, wj, Qj, Qm);
            const bool self = (sm == sj) && (j2m == j2);
            buf[sj * P2 + j2] = Qj;
            if (!self) buf[sm * P2 + j2m] = Qm;
            if (two) {
                repack_pair(al2, be2, wj, Qj, Qm);
                buf2[sj * P2 + j2] = Qj;
                if (!self) buf2[sm * P2 + j2m] = Qm;
            }
        }
        __syncthreads();
        fft_inplace<W, Ept<W>::v, true>(buf, A.logP2, two ? 2 * nrows : nrows, P2, tw, I.logTW);
        for (int idx = threadIdx.x; idx < nrows * P2; idx += blockDim.x) {
            const int sl = idx / P2, m2 = idx - sl * P2;
            const cx<W> w = conj(tw[(rows[sl] * m2) << tsh]);
            Y[(long long)rows[sl] * P2 + m2] = buf[idx] * w;
            if (two) Y2[(long long)rows[sl] * P2 + m2] = buf2[idx] * w;
        }
        __syncthreads();
    }
}

// Column phase of the inverse transform: P1-point inverse FFTs of columns
// of Y (and Y2), unpack q_m -> a_{2m}, a_{2m+1}, epilogue.
template <typename W, bool TWO, typename EpiF>
FDE_NI void split_inv_cols(const Team& t, const Inst& I, const cx<W>* Y, const cx<W>* Y2, unsigned char* work,
                          int cc, EpiF epi) {
    const AxisData& A = I.ax[0];
    const int n = A.n, P1 = A.P1, P2 = A.P2;
    const cx<W>* tw = Prec<W>::tw(I);
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    cx<W>* buf2 = buf + cc * P1;
    const int units = P2 / cc;
    for (int u = t.rank; u < units; u += t.size) {
        const int m2b = u * cc;
        for (int idx = threadIdx.x; idx < cc * P1; idx += blockDim.x) {
            const int c = idx % cc, j1 = idx / cc;
            buf[c * P1 + j1] = ldw(Y + (long long)j1 * P2 + m2b + c);
            if (TWO) buf2[c * P1 + j1] = ldw(Y2 + (long long)j1 * P2 + m2b + c);
        }
        __syncthreads();
        fft_inplace<W, Ept<W>::v, true>(buf, A.logP1, TWO ? 2 * cc : cc, P1, tw, I.logTW);
        for (int idx = threadIdx.x; idx < cc * P1; idx += blockDim.x) {
            const int c = idx % cc, m1 = idx / cc;
            const long long m = (long long)P2 * m1 + m2b + c;
            const cx<W> q = buf[c * P1 + m1];
            const cx<W> q2 = TWO ? buf2[c * P1 + m1] : czero<W>();
            const long long k0 = 2 * m, k1 = 2 * m + 1;       // a_k for k = 1..n
            if (k0 >= 1 && k0 <= n) epi(k0 - 1, q.x, q2.x);
            if (k1 <= n) epi(k1 - 1, q.y, q2.y);
        }
        __syncthreads();
    }
}

template <typename W>
FDE_NI bool split_matvec_1d(const Team& t, const Inst& I, const W* x, W s, W* y, unsigned char* work, int bytes) {
    const AxisData& A = I.ax[0];
    const bool sym = I.symx;
    cx<W>* Y = Prec<W>::split(I);
    cx<W>* Y2 = Y + A.Np;
    const RealIn<W> in{x, 1, s, nullptr};
    const int cc1 = split_cols_per_unit<W>(A, t.size, 1, bytes);
    split_fwd_cols<W, kExtZero>(t, I, in, Y, work, cc1);
    if (!team_sync(t)) return false;
    split_rows<W>(t, I, mult_matvec<W>(A, sym), Y, Y2, work);
    if (!team_sync(t)) return false;
    const W c0s = W(I.c0) * s;
    const W* dp = Prec<W>::dp(I);
    const W* dm = Prec<W>::dm(I);
    if (sym) {
        split_inv_cols<W, false>(t, I, Y, Y2, work, cc1, [&](long long p, W va, W) {
            y[p] = c0s * ldw(x + p) + coef(dp, I.dpc, p) * va;
        });
    } else {
        const int cc2 = split_cols_per_unit<W>(A, t.size, 2, bytes);
        split_inv_cols<W, true>(t, I, Y, Y2, work, cc2, [&](long long p, W va, W vb) {
            y[p] = c0s * ldw(x + p) + coef(dp, I.dpc, p) * va + coef(dm, I.dmc, p) * vb;
        });
    }
    return true;
}

template <typename W>
FDE_NI bool split_tau_1d(const Team& t, const Inst& I, const W* r, W s, W* z, unsigned char* work, int bytes) {
    const AxisData& A = I.ax[0];
    cx<W>* Y = Prec<W>::split(I);
    const W* dinv = Prec<W>::dinv(I);
    const bool pre = I.has_D && I.order == FDE_ORDER_D_TAU;
    const bool post = I.has_D && I.order == FDE_ORDER_TAU_D;
    const RealIn<W> in{r, 1, s, pre ? dinv : nullptr};
    const int cc = split_cols_per_unit<W>(A, t.size, 1, bytes);
    split_fwd_cols<W, kExtOdd>(t, I, in, Y, work, cc);
    if (!team_sync(t)) return false;
    split_rows<W>(t, I, mult_tau1<W>(A), Y, nullptr, work);
    if (!team_sync(t)) return false;
    split_inv_cols<W, false>(t, I, Y, nullptr, work, cc, [&](long long p, W va, W) {
        z[p] = post ? va * __ldg(dinv + p) : va;
    });
    return true;
}

// ---------------------------------------------------------------------------
// 2D plane: rows (x lines, contiguous) and columns (y lines, stride n1)
// ---------------------------------------------------------------------------

template <typename W>
FDE_D int plane_lines_per_unit(int Np, int nbuf, int nlines_total, int team_size, int bytes, int extra_real) {
    // extra_real: bytes of a real Np-array per line kept beside the buffers
    int cap = max_lines<W>(Np, nbuf, bytes - 64);
    if (extra_real) {
        const int per = (int)(Np * (nbuf * sizeof(cx<W>) + sizeof(W)));
        const int c2 = bytes / per;
        if (c2 < cap) cap = c2;
    }
    int want = (nlines_total + team_size - 1) / team_size;
    int b = want < cap ? want : cap;
    if (b < 1) b = 1;
    return b;
}

// Lone DST-I along rows: out[row, j-1] = s_j of (scale * in[row, :]) (* pre),
// multiplied by post[row, j-1] when post != null.
template <typename W>
FDE_NI void plane_dst_rows(const Team& t, const Inst& I, const W* in, W s, const W* pre, const W* post, W* out,
                          unsigned char* work, int bytes) {
    const AxisData& A = I.ax[0];
    const int n1 = A.n, Np = A.Np, n2 = I.n2;
    const int B = plane_lines_per_unit<W>(Np, 1, n2, t.size, bytes, 1);
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    W* sv = reinterpret_cast<W*>(buf + B * Np);
    const int units = (n2 + B - 1) / B;
    for (int u = t.rank; u < units; u += t.size) {
        const int row0 = u * B;
        const int nb = (n2 - row0) < B ? (n2 - row0) : B;
        cta_pack<W, kExtOdd, false>(buf, nb, n1, Np, [&](int l) {
            const long long o = (long long)(row0 + l) * n1;
            return RealIn<W>{in + o, 1, s, pre ? pre + o : nullptr};
        });
        fft_inplace<W, Ept<W>::v, false>(buf, A.logNp, nb, Np, Prec<W>::tw(I), I.logTW);
        cta_dst_extract<W>(buf, sv, nb, Np, A.logNp, Prec<W>::tw(I), I.logTW);
        for (int idx = threadIdx.x; idx < nb * n1; idx += blockDim.x) {
            const int l = idx / n1, p = idx - l * n1;
            const long long o = (long long)(row0 + l) * n1 + p;
            W v = sv[l * Np + p + 1];
            if (post) v *= __ldg(post + o);
            out[o] = v;
        }
        __syncthreads();
    }
}

// tau^{-1} along columns in place: z[:, c] <- S2 diag(phi) S2 z[:, c].
template <typename W>
FDE_NI void plane_tau_cols(const Team& t, const Inst& I, W* z, unsigned char* work, int bytes) {
    const AxisData& A = I.ax[1];
    const int n2 = A.n, Np = A.Np, n1 = I.n1;
    const int C = plane_lines_per_unit<W>(Np, 1, n1, t.size, bytes, 0);
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    const Mult<W> mu = mult_tau2<W>(I);
    const int units = (n1 + C - 1) / C;
    for (int u = t.rank; u < units; u += t.size) {
        const int c0 = u * C;
        const int nc = (n1 - c0) < C ? (n1 - c0) : C;
        cta_pack<W, kExtOdd, true>(buf, nc, n2, Np, [&](int l) {
            return RealIn<W>{z + c0 + l, n1, W(1), nullptr};
        });
        fft_inplace<W, Ept<W>::v, false>(buf, A.logNp, nc, Np, Prec<W>::tw(I), I.logTW);
        cta_spectral<W>(buf, nullptr, nc, Np, A.logNp, Prec<W>::tw(I), I.logTW, mu,
                        [&](int l) { return c0 + l; });
        fft_inplace<W, Ept<W>::v, true>(buf, A.logNp, nc, Np, Prec<W>::tw(I), I.logTW);
        cta_unpack<W, true, false>(buf, nullptr, nc, n2, Np, [&](int l, int p, W va, W) {
            z[(long long)p * n1 + c0 + l] = va;
        });
        __syncthreads();
    }
}

// x part of the matvec: tmp = c0 s x + D_+ (I (x) T_a)(s x) + D_- (I (x) T_a^T)(s x).
template <typename W>
FDE_NI void plane_matvec_rows(const Team& t, const Inst& I, const W* x, W s, W* tmp, unsigned char* work,
                             int bytes) {
    const AxisData& A = I.ax[0];
    const int n1 = A.n, Np = A.Np, n2 = I.n2;
    const bool sym = I.symx;
    const int B = plane_lines_per_unit<W>(Np, sym ? 1 : 2, n2, t.size, bytes, 0);
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    const Mult<W> mu = mult_matvec<W>(A, sym);
    const W c0s = W(I.c0) * s;
    const W* dp = Prec<W>::dp(I);
    const W* dm = Prec<W>::dm(I);
    const int units = (n2 + B - 1) / B;
    for (int u = t.rank; u < units; u += t.size) {
        const int row0 = u * B;
        const int nb = (n2 - row0) < B ? (n2 - row0) : B;
        cx<W>* buf2 = buf + nb * Np;
        cta_pack<W, kExtZero, false>(buf, nb, n1, Np, [&](int l) {
            return RealIn<W>{x + (long long)(row0 + l) * n1, 1, s, nullptr};
        });
        fft_inplace<W, Ept<W>::v, false>(buf, A.logNp, nb, Np, Prec<W>::tw(I), I.logTW);
        cta_spectral<W>(buf, buf2, nb, Np, A.logNp, Prec<W>::tw(I), I.logTW, mu, [](int) { return 0; });
        fft_inplace<W, Ept<W>::v, true>(buf, A.logNp, sym ? nb : 2 * nb, Np, Prec<W>::tw(I), I.logTW);
        if (sym) {
            cta_unpack<W, false, false>(buf, buf2, nb, n1, Np, [&](int l, int p, W va, W) {
                const long long o = (long long)(row0 + l) * n1 + p;
                tmp[o] = c0s * ldw(x + o) + coef(dp, I.dpc, o) * va;
            });
        } else {
            cta_unpack<W, false, true>(buf, buf2, nb, n1, Np, [&](int l, int p, W va, W vb) {
                const long long o = (long long)(row0 + l) * n1 + p;
                tmp[o] = c0s * ldw(x + o) + coef(dp, I.dpc, o) * va + coef(dm, I.dmc, o) * vb;
            });
        }
        __syncthreads();
    }
}

// y part: y = tmp + sr [E_+ (T_b (x) I)(s x) + E_- (T_b^T (x) I)(s x)].
template <typename W>
FDE_NI void plane_matvec_cols(const Team& t, const Inst& I, const W* x, W s, const W* tmp, W* y,
                             unsigned char* work, int bytes) {
    const AxisData& A = I.ax[1];
    const int n2 = A.n, Np = A.Np, n1 = I.n1;
    const bool sym = I.symy;
    const int C = plane_lines_per_unit<W>(Np, sym ? 1 : 2, n1, t.size, bytes, 0);
    cx<W>* buf = reinterpret_cast<cx<W>*>(work);
    const Mult<W> mu = mult_matvec<W>(A, sym);
    const W sr = W(I.sr);
    const W* ep = Prec<W>::ep(I);
    const W* em = Prec<W>::em(I);
    const int units = (n1 + C - 1) / C;
    for (int u = t.rank; u < units; u += t.size) {
        const int c0 = u * C;
        const int nc = (n1 - c0) < C ? (n1 - c0) : C;
        cx<W>* buf2 = buf + nc * Np;
        cta_pack<W, kExtZero, true>(buf, nc, n2, Np, [&](int l) {
            return RealIn<W>{x + c0 + l, n1, s, nullptr};
        });
        fft_inplace<W, Ept<W>::v, false>(buf, A.logNp, nc, Np, Prec<W>::tw(I), I.logTW);
        cta_spectral<W>(buf, buf2, nc, Np, A.logNp, Prec<W>::tw(I), I.logTW, mu, [](int) { return 0; });
        fft_inplace<W, Ept<W>::v, true>(buf, A.logNp, sym ? nc : 2 * nc, Np, Prec<W>::tw(I), I.logTW);
        if (sym) {
            cta_unpack<W, true, false>(buf, buf2, nc, n2, Np, [&](int l, int p, W va, W) {
                const long long o = (long long)p * n1 + c0 + l;
                y[o] = ldw(tmp + o) + sr * coef(ep, I.epc, o) * va;
            });
        } else {
            cta_unpack<W, true, true>(buf, buf2, nc, n2, Np, [&](int l, int p, W va, W vb) {
                const long long o = (long long)p * n1 + c0 + l;
                y[o] = ldw(tmp + o) + sr * (coef(ep, I.epc, o) * va + coef(em, I.emc, o) * vb);
            });
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Dispatch.  `tmp` is an N-vector of scratch (2D matvec only).
// ---------------------------------------------------------------------------

template <typename W>
FDE_D bool op_matvec(const Team& t, const Inst& I, int line_mode, const W* x, W s, W* y, W* tmp,
                     unsigned char* work, int bytes) {
    if (I.dim == 1) {
        if (line_mode == kLineCta) {
            if (t.rank == 0) cta_matvec_1d<W>(I, x, s, y, work);
        } else {
            if (!split_matvec_1d<W>(t, I, x, s, y, work, bytes)) return false;
        }
    } else {
        plane_matvec_rows<W>(t, I, x, s, tmp, work, bytes);
        if (!team_sync(t)) return false;
        plane_matvec_cols<W>(t, I, x, s, tmp, y, work, bytes);
    }
    return team_sync(t);
}

template <typename W>
FDE_D bool op_tau(const Team& t, const Inst& I, int line_mode, const W* r, W s, W* z, unsigned char* work,
                  int bytes) {
    if (I.dim == 1) {
        if (line_mode == kLineCta) {
            if (t.rank == 0) cta_tau_1d<W>(I, r, s, z, work);
        } else {
            if (!split_tau_1d<W>(t, I, r, s, z, work, bytes)) return false;
        }
    } else {
        const W* dinv = Prec<W>::dinv(I);
        const bool pre = I.has_D && I.order == FDE_ORDER_D_TAU;
        const bool post = I.has_D && I.order == FDE_ORDER_TAU_D;
        plane_dst_rows<W>(t, I, r, s, pre ? dinv : nullptr, nullptr, z, work, bytes);
        if (!team_sync(t)) return false;
        plane_tau_cols<W>(t, I, z, work, bytes);
        if (!team_sync(t)) return false;
        plane_dst_rows<W>(t, I, z, W(1), nullptr, post ? dinv : nullptr, z, work, bytes);
    }
    return team_sync(t);
}

}  // namespace fde
