// Line transforms of the two operators, built on the real-packed FFT.
//
// A real line r_1..r_n (n = Np - 1) is extended to length L = 2 Np either by
// zeros (Toeplitz product by circulant embedding) or oddly (DST-I, Sec. 1:
// v_0 = v_Np = 0, v_{L-k} = -r_k).  The extension is packed into Np complex
// values z_m = v_{2m} + i v_{2m+1} and transformed with an Np-point FFT; the
// L-point spectrum follows from the pairs (Z_j, Z_{Np-j}):
//   E_j = (Z_j + conj Z_{Np-j})/2,  O_j = (Z_j - conj Z_{Np-j})/(2i),
//   X_j = E_j + w_L^j O_j,  X_{j+Np} = E_j - w_L^j O_j.
// A Hermitian multiplier mu (mu_{L-k} = conj mu_k) keeps the inverse real:
//   A_j = mu_j X_j, A_{j+Np} = conj(mu_{Np-j}) X_{j+Np},
//   Q_j = (A_j + A_{j+Np}) + i w_L^{-j} (A_j - A_{j+Np}),
// and the Np-point inverse FFT of Q gives a_{2m} + i a_{2m+1}.
//
// Operators (multipliers are stored pre-divided by L):
//   T x      : mu = lambda  (eigenvalues of the circulant embedding T)
//   T^T x    : mu = conj(lambda)
//   (T+T^T)x : mu = 2 Re(lambda)
//   tau^{-1} : mu = 1/(L F(theta_k)) on the odd extension, which equals
//              S diag(1/F) S (the two sine transforms of Sec. 1)
//   S r      : the odd-extension spectrum itself, S r = sqrt(2/Np) (-Im X_j / 2)
//
// Shared-memory line buffers hold lines at stride Np in a flat index space
// and are accessed through pad(); a second output set (kMulLam2) occupies
// the lines that follow the first set.
#pragma once

#include "fft.cuh"
#include "team.cuh"

namespace fde {

enum Ext : int { kExtZero = 0, kExtOdd = 1 };

// Loads of data that other CTAs of the team wrote in an earlier phase go
// through L2 only (ld.global.cg), never a possibly stale L1 line.
template <typename W>
FDE_D W ldw(const W* p) { return __ldcg(p); }
FDE_D cx<double> ldw(const cx<double>* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mk(v.x, v.y);
}
FDE_D cx<float> ldw(const cx<float>* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return mk(v.x, v.y);
}

// v_k of the length-L extension of a line.  get(k, direct) returns r_k
// (1 <= k <= n); `direct` is true for exactly one read of every r_k (the
// unmirrored one), so a getter may store or accumulate there.
template <typename W, int EXT, typename GetF>
FDE_D W ext_val(GetF& get, int k, int n, int Np) {
    if (k >= 1 && k <= n) return get(k, true);
    if (EXT == kExtOdd && k > Np) return -get(2 * Np - k, false);
    return W(0);
}

template <typename W, int EXT, typename GetF>
FDE_D cx<W> pack_elem(GetF& get, int m, int n, int Np) {
    return mk(ext_val<W, EXT>(get, 2 * m, n, Np), ext_val<W, EXT>(get, 2 * m + 1, n, Np));
}

template <typename R>
FDE_D void unpack_pair(cx<R> Zj, cx<R> Zm, cx<R> wj, cx<R>& a, cx<R>& b) {
    const cx<R> Zc = conj(Zm);
    const cx<R> E = R(0.5) * (Zj + Zc);
    const cx<R> O = mul_mi(R(0.5) * (Zj - Zc));
    const cx<R> t = wj * O;
    a = E + t;
    b = E - t;
}

template <typename R>
FDE_D void repack_pair(cx<R> al, cx<R> be, cx<R> wj, cx<R>& Qj, cx<R>& Qm) {
    const cx<R> s = al + be, d = al - be;
    Qj = s + mul_i(conj(wj) * d);
    Qm = conj(s) + mul_i(wj * conj(d));
}

// Multiplier kinds for the spectral step.
enum MulKind : int { kMulLam2 = 0, kMulSym = 1, kMulTau1 = 2, kMulTau2 = 3 };

template <typename W>
struct Mult {
    int kind;
    const cx<W>* lam;      // [Np+1]
    const W* phi;          // kMulTau1: [Np+1] multiplier; kMulTau2: [Np+1] y-axis symbol part
    const W* a1;           // kMulTau2: x-axis symbol part, indexed by x-frequency
    W scale2d;             // kMulTau2: 2/(n1+1)/L2
    int n, Np;

    // Multipliers for the pair (j, Np - j): first output and, for kMulLam2,
    // the second (conj(lambda)).  `col` is the x-frequency index for kMulTau2.
    FDE_D void apply(int j, int col, cx<W> a, cx<W> b, cx<W>& al, cx<W>& be, cx<W>& al2,
                     cx<W>& be2) const {
        const int jm = Np - j;
        if (kind == kMulLam2) {
            const cx<W> lj = lam[j];
            const cx<W> lm = lam[jm];
            al = lj * a;
            be = conj(lm) * b;
            al2 = conj(lj) * a;
            be2 = lm * b;
        } else if (kind == kMulSym) {
            al = (W(2) * lam[j].x) * a;
            be = (W(2) * lam[jm].x) * b;
        } else if (kind == kMulTau1) {
            al = phi[j] * a;
            be = phi[jm] * b;
        } else {
            const W ax = a1[col + 1];
            const W pj = (j >= 1 && j <= n) ? scale2d / (ax + phi[j]) : W(0);
            const W pm = (jm >= 1 && jm <= n) ? scale2d / (ax + phi[jm]) : W(0);
            al = pj * a;
            be = pm * b;
        }
    }
};

// ---------------------------------------------------------------------------
// Whole lines held by one CTA: B lines of Np complex values, flat index
// l * Np + m through pad().
// ---------------------------------------------------------------------------

// Position (l, m) of element idx of B lines of Np points (Np a power of two),
// idx = l Np + m (ROW) or m B + l (COLMAJOR: consecutive threads on
// consecutive lines, coalesced for strided columns), advanced by a fixed
// step without a division per element.
struct Walk {
    int l, m, dl, dm, B, Np;
    FDE_D Walk(bool colmajor, int start, int step, int B_, int logNp) : B(B_), Np(1 << logNp) {
        if (colmajor) { l = start % B; m = start / B; dl = step % B; dm = step / B; }
        else { l = start >> logNp; m = start & (Np - 1); dl = step >> logNp; dm = step & (Np - 1); }
    }
    FDE_D void next(bool colmajor) {
        l += dl;
        m += dm;
        if (colmajor) { if (l >= B) { l -= B; ++m; } }
        else if (m >= Np) { m -= Np; ++l; }
    }
};

FDE_D int log2_pow2(int v) { return 31 - __clz(v); }

// Pack B real lines.  get(l, k, direct) returns r_k of line l.
// Each thread gathers kPackUnroll elements before storing any, so their global
// loads are in flight together (the getters only load); an unpack holds the
// operands of kUnpackUnroll elements.
template <typename W> constexpr int kPackUnroll = sizeof(W) == 4 ? 8 : 4;
constexpr int kUnpackUnroll = 4;

template <typename W, int EXT, bool COLMAJOR, typename GetF>
FDE_D void cta_pack(const Grp& g, cx<W>* buf, int B, int n, int Np, GetF get) {
    constexpr int kUnroll = kPackUnroll<W>;
    const int logNp = log2_pow2(Np);
    const int total = B << logNp;
    const int nt = g.nt;
    Walk w(COLMAJOR, g.tid, nt, B, logNp);
    for (int base = g.tid; base < total; base += kUnroll * nt) {
        cx<W> v[kUnroll];
        int at[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            at[u] = -1;
            if (base + u * nt < total) {
                const int l = w.l, m = w.m;
                auto g = [&](int k, bool direct) { return get(l, k, direct); };
                v[u] = pack_elem<W, EXT>(g, m, n, Np);
                at[u] = (l << logNp) + m;
            }
            w.next(COLMAJOR);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (at[u] >= 0) buf[pad(at[u])] = v[u];
    }
    grp_sync(g);
}

// Pairs (j, Np - j) of B lines, j = 0..Np/2: f(l, j) per pair, no division
// per pair (Np >= 2, a power of two).
template <typename F>
FDE_D void cta_pairs(const Grp& g, int B, int logNp, F f) {
    const int lh = logNp - 1;
    const int hm = 1 << lh;
    const int total = B << lh;
    for (int idx = g.tid; idx < total + B; idx += g.nt) {
        if (idx < total) f(idx >> lh, idx & (hm - 1));
        else f(idx - total, hm);
    }
}

// Spectral step on all pairs of B lines; the second output (kMulLam2) goes
// to lines B..2B-1.  col_of_line gives kMulTau2's x-frequency of a line.
template <typename W, typename ColF>
FDE_D void cta_spectral(const Grp& g, cx<W>* buf, int B, int Np, int logNp, const Tw& tw, const Mult<W>& mu,
                        ColF col_of_line) {
    const bool two = mu.kind == kMulLam2;
    cta_pairs(g, B, logNp, [&](int l, int j) {
        const int jm = (Np - j) & (Np - 1);
        const int o = l * Np;
        const cx<W> wj = tw_L<W>(tw, j, logNp + 1);
        cx<W> a, b, al, be, al2, be2;
        unpack_pair(buf[pad(o + j)], buf[pad(o + jm)], wj, a, b);
        mu.apply(j, col_of_line(l), a, b, al, be, al2, be2);
        cx<W> Qj, Qm;
        repack_pair(al, be, wj, Qj, Qm);
        buf[pad(o + j)] = Qj;
        if (jm != j) buf[pad(o + jm)] = Qm;
        if (two) {
            const int o2 = (B + l) * Np;
            repack_pair(al2, be2, wj, Qj, Qm);
            buf[pad(o2 + j)] = Qj;
            if (jm != j) buf[pad(o2 + jm)] = Qm;
        }
    });
    grp_sync(g);
}

// Lone DST-I of B lines: after the forward FFT of the odd extension, write
// the unnormalised sine sums s_j = -Im X_j / 2 (j = 1..n) into the real
// shared-memory array s (B lines at stride Np, unpadded).
template <typename W>
FDE_D void cta_dst_extract(const Grp& g, const cx<W>* buf, W* s, int B, int Np, int logNp, const Tw& tw) {
    cta_pairs(g, B, logNp, [&](int l, int j) {
        const int jm = (Np - j) & (Np - 1);
        const int o = l * Np;
        cx<W> a, b;
        unpack_pair(buf[pad(o + j)], buf[pad(o + jm)], tw_L<W>(tw, j, logNp + 1), a, b);
        if (j >= 1) {
            s[o + j] = W(-0.5) * a.y;
            if (jm != j) s[o + (Np - j)] = W(0.5) * b.y;
        }
    });
    grp_sync(g);
}

// Forward FFT of B lines, the spectral step with mu (kMulTau2's x-frequency
// of line l is col0 + l) and the inverse FFT of the nout output lines, in
// one call: the register saves of a non-inlined call are paid once per unit
// of lines instead of once per transform.
template <typename W>
FDE_NI void fft_spectral_lines(const Grp g, cx<W>* buf, int B, int Np, int logNp, const Tw& tw, const Mult<W>& mu,
                               int col0, int nout) {
    fft_lines_in<W, false>(g, buf, logNp, B, Np, tw);
    cta_spectral<W>(g, buf, B, Np, logNp, tw, mu, [&](int l) { return col0 + l; });
    fft_lines_in<W, true>(g, buf, logNp, nout, Np, tw);
}

// Forward FFT of the odd extensions of B lines and the sine sums s_j, in one
// call.
template <typename W>
FDE_NI void fft_dst_lines(const Grp g, cx<W>* buf, W* s, int B, int Np, int logNp, const Tw& tw) {
    fft_lines_in<W, false>(g, buf, logNp, B, Np, tw);
    cta_dst_extract<W>(g, buf, s, B, Np, logNp, tw);
}

// Unpack q_m = a_{2m} + i a_{2m+1} and hand a_k (k = 1..n, p = k - 1) to
// put(l, p, a_k, b_k, fetch(l, p)), b from the second output set when TWO.
// The fetches of kUnpackUnroll elements (the epilogue's global loads) are issued
// before any of their puts, so the loads are in flight together.
template <typename W, bool COLMAJOR, bool TWO, typename FetchF, typename PutF>
FDE_D void cta_unpack2(const Grp& g, const cx<W>* buf, int B, int n, int Np, FetchF fetch, PutF put) {
    constexpr int kUnroll = kUnpackUnroll;
    const int logNp = log2_pow2(Np);
    const int total = B << logNp;
    const int nt = g.nt;
    Walk w(COLMAJOR, g.tid, nt, B, logNp);
    using Ops = decltype(fetch(0, 0));
    for (int base = g.tid; base < total; base += kUnroll * nt) {
        Ops ops[kUnroll];
        W va[kUnroll], vb[kUnroll];
        int li[kUnroll], pi[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            li[u] = -1;
            const int l = w.l, p = w.m;
            if (base + u * nt < total && p < n) {
                li[u] = l;
                pi[u] = p;
                ops[u] = fetch(l, p);
                const int k = p + 1;
                const cx<W> q = buf[pad(l * Np + (k >> 1))];
                va[u] = (k & 1) ? q.y : q.x;
                vb[u] = W(0);
                if (TWO) {
                    const cx<W> q2 = buf[pad((B + l) * Np + (k >> 1))];
                    vb[u] = (k & 1) ? q2.y : q2.x;
                }
            }
            w.next(COLMAJOR);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (li[u] >= 0) put(li[u], pi[u], va[u], vb[u], ops[u]);
    }
}

struct NoOps {};

// Unpack with an epilogue that loads nothing: epi(l, p, a_k, b_k).
template <typename W, bool COLMAJOR, bool TWO, typename EpiF>
FDE_D void cta_unpack(const Grp& g, const cx<W>* buf, int B, int n, int Np, EpiF epi) {
    cta_unpack2<W, COLMAJOR, TWO>(g, buf, B, n, Np, [](int, int) { return NoOps{}; },
                                  [&](int l, int p, W va, W vb, const NoOps&) { epi(l, p, va, vb); });
}

}  // namespace fde
