// The two operators of one Krylov iteration, for every data layout:
//   op_matvec: y = M (s x)      (Sec. 1.2 / 1.4, Toeplitz by circulant embedding)
//   op_tau:    z = P^{-1} (s r) (Sec. 3.1 / 3.2, DST-I / symbol / DST-I)
// and the phases that the fused right-preconditioned Arnoldi step combines.
//
// Layouts: a 1D line held whole by one CTA; a 1D line split across the CTAs
// of a team (Np = P1 * P2: column / row / column phases through an
// L2-resident intermediate Y); a 2D plane (row lines along x, column lines
// along y).  Phase functions take a getter for their input (so a basis
// vector can be formed on the fly) and an epilogue for their output.
#pragma once

#include "lines.cuh"

namespace fde {

template <typename W>
FDE_D W coef(const W* arr, double cst, long long i) {
    return arr ? __ldg(arr + i) : W(cst);
}

// Shared memory and twiddles of one CTA for transform phases.
struct Wk {
    unsigned char* smem;
    int bytes;
    Tw tw;
};

// Lines of Np complex values (nbuf buffers each, padded) plus `extra_real`
// real arrays of Np per line that fit `bytes` of shared memory.
template <typename W>
FDE_HD int max_lines(int Np, int nbuf, int bytes, int extra_real = 0) {
    const long long per = (long long)Np * nbuf * sizeof(cx<W>) * 17 / 16 + (long long)Np * extra_real * sizeof(W) + 16;
    return (int)((bytes - 64) / per);
}

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
// Inputs formed on the fly: u_p = s * (base_p - sum_q c_q V_q[p]) where V_q
// are vectors at stride N (the solution update of GMRES combines its basis
// this way).
// ---------------------------------------------------------------------------

// A phase's multipliers in a per-CTA shared slot, for the fused transform
// calls (a reference to a thread-local copy would be a stack address, read
// back through the small L1 beside the work area).  Every thread of the CTA
// calls this at the start of a phase.
template <typename W>
FDE_D const Mult<W>& mult_slot(const Mult<W>& m) {
    __shared__ Mult<W> s;
    __syncthreads();
    if (threadIdx.x == 0) s = m;
    __syncthreads();
    return s;
}

template <typename W>
struct Combo {
    const W* base;         // may be null (then 0)
    const W* V;
    const W* c;            // shared memory, cnt coefficients (working precision)
    int cnt;
    long long N;
    W s;
    const W* pre;          // optional elementwise prescale applied after s (D^{-1} for P = D tau)

    // In the working precision: a basis update is a vector operation, not an
    // inner product.
    FDE_D W raw(long long p) const {
        W v = base ? ldw(base + p) : W(0);
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) v -= c[q] * ldw(V + (long long)q * N + p);
        return v;
    }
    FDE_D W get(long long p, bool) const {
        W v = s * raw(p);
        if (pre) v *= __ldg(pre + p);
        return v;
    }
};

template <typename W>
FDE_D Combo<W> combo_vec(const W* x, W s, const W* pre = nullptr) {
    Combo<W> c{};
    c.base = x;
    c.s = s;
    c.pre = pre;
    return c;
}


// ---------------------------------------------------------------------------
// Epilogues.  A transform hands (a, b) per element (b: the second product of
// a two-multiplier matvec); the epilogue forms the value and writes it.
// ---------------------------------------------------------------------------

enum ValKind : int { kValA = 0, kValMvX = 1, kValMvY = 2 };
enum OutKind : int { kOutStore = 0, kOutResid = 1, kOutAdd = 2 };

// Where a result goes: out = v, out = rhs - v, or out += v.
template <typename W>
struct OutSpec {
    int outk;
    W* out;
    const W* rhs;
};

template <typename W>
FDE_D OutSpec<W> out_store(W* out) { return OutSpec<W>{kOutStore, out, nullptr}; }

template <typename W>
struct Epi {
    int val;               // kValA: a (* post); kValMvX: c0 s x + c+ a + c- b; kValMvY: tmp + sr (c+ a + c- b)
    OutSpec<W> o;
    const W* post;
    const W* x;
    W xs, c0, sr;
    const W* cp;
    const W* cm;
    double cpc, cmc;
    int sym;
    const W* tmp;

    // The operands of element p, loaded (fetch) apart from the arithmetic and
    // the store (put), so that a caller can have the loads of several
    // elements in flight before it stores any.
    struct Ops {
        W x, c1, c2, o;
    };
    FDE_D Ops fetch(long long p) const {
        Ops r;
        r.x = r.c1 = r.c2 = r.o = W(0);
        if (val == kValA) {
            r.c1 = post ? __ldg(post + p) : W(1);
        } else {
            r.c1 = cp ? __ldg(cp + p) : W(cpc);
            if (!sym) r.c2 = cm ? __ldg(cm + p) : W(cmc);
            r.x = ldw((val == kValMvX ? x : tmp) + p);
        }
        if (o.outk == kOutResid) r.o = ldw(o.rhs + p);
        else if (o.outk == kOutAdd) r.o = o.out[p];
        return r;
    }
    FDE_D void put(long long p, W a, W b, const Ops& r) const {
        W v;
        if (val == kValA) {
            v = post ? a * r.c1 : a;
        } else {
            W t = r.c1 * a;
            if (!sym) t += r.c2 * b;
            v = val == kValMvX ? c0 * xs * r.x + t : r.x + sr * t;
        }
        if (o.outk == kOutStore) o.out[p] = v;
        else if (o.outk == kOutResid) o.out[p] = r.o - v;
        else o.out[p] = r.o + v;
    }
    FDE_D void operator()(long long p, W a, W b) const { put(p, a, b, fetch(p)); }
};

template <typename W>
FDE_D Epi<W> epi_a(const W* post, OutSpec<W> o) {
    Epi<W> e{};
    e.val = kValA;
    e.post = post;
    e.o = o;
    return e;
}

// x part (1D: the whole matvec): c0 s x + D_+ a + D_- b.
template <typename W>
FDE_D Epi<W> epi_mvx(const Inst& I, const W* x, W s, OutSpec<W> o) {
    Epi<W> e{};
    e.val = kValMvX;
    e.o = o;
    e.x = x;
    e.xs = s;
    e.c0 = W(I.c0);
    e.cp = Prec<W>::dp(I);
    e.cm = Prec<W>::dm(I);
    e.cpc = I.dpc;
    e.cmc = I.dmc;
    e.sym = I.symx;
    return e;
}

// y part (2D): tmp + sr (E_+ a + E_- b).
template <typename W>
FDE_D Epi<W> epi_mvy(const Inst& I, const W* tmp, OutSpec<W> o) {
    Epi<W> e{};
    e.val = kValMvY;
    e.o = o;
    e.tmp = tmp;
    e.sr = W(I.sr);
    e.cp = Prec<W>::ep(I);
    e.cm = Prec<W>::em(I);
    e.cpc = I.epc;
    e.cmc = I.emc;
    e.sym = I.symy;
    return e;
}

// ---------------------------------------------------------------------------
// 1D, whole line in one CTA (team of one)
// ---------------------------------------------------------------------------

// z = tau^{-1}(u); epi(p, z_p).  D^{-1} per the order is applied here.
template <typename W>
FDE_NI void cta_tau_1d(const Inst& I, const Wk& wk, Combo<W> u, Epi<W> epi) {
    const AxisData& A = I.ax[0];
    const int n = A.n, Np = A.Np;
    cx<W>* buf = reinterpret_cast<cx<W>*>(wk.smem);
    const W* dinv = Prec<W>::dinv(I);
    if (I.has_D && I.order == FDE_ORDER_D_TAU) u.pre = dinv;
    if (I.has_D && I.order == FDE_ORDER_TAU_D) epi.post = dinv;
    const Mult<W>& mu = mult_slot<W>(mult_tau1<W>(A));
    cta_pack<W, kExtOdd, false>(grp_cta(), buf, 1, n, Np, [&](int, int k, bool d) { return u.get(k - 1, d); });
    fft_spectral_lines<W>(grp_cta(), buf, 1, Np, A.logNp, wk.tw, mu, 0, 1);
    cta_unpack2<W, false, false>(grp_cta(), buf, 1, n, Np, [&](int, int p) { return epi.fetch(p); },
                                 [&](int, int p, W va, W vb, const typename Epi<W>::Ops& r) { epi.put(p, va, vb, r); });
    __syncthreads();
}

// the matvec of s x; epi(p, (T x)_p, (T^T x)_p) -- symmetric: ((T+T^T) x)_p.
template <typename W>
FDE_NI void cta_matvec_1d(const Inst& I, const Wk& wk, const W* x, W s, Epi<W> epi) {
    const AxisData& A = I.ax[0];
    const int n = A.n, Np = A.Np;
    cx<W>* buf = reinterpret_cast<cx<W>*>(wk.smem);
    const bool sym = I.symx;
    const Mult<W>& mu = mult_slot<W>(mult_matvec<W>(A, sym));
    cta_pack<W, kExtZero, false>(grp_cta(), buf, 1, n, Np, [&](int, int k, bool) { return s * ldw(x + (k - 1)); });
    fft_spectral_lines<W>(grp_cta(), buf, 1, Np, A.logNp, wk.tw, mu, 0, sym ? 1 : 2);
    auto fe = [&](int, int p) { return epi.fetch(p); };
    auto pu = [&](int, int p, W va, W vb, const typename Epi<W>::Ops& r) { epi.put(p, va, vb, r); };
    if (sym) cta_unpack2<W, false, false>(grp_cta(), buf, 1, n, Np, fe, pu);
    else cta_unpack2<W, false, true>(grp_cta(), buf, 1, n, Np, fe, pu);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// P_tri (Sec. 4, Table 2): z = P^{-1} u for the tridiagonal part of M by
// parallel cyclic reduction.  A round with stride s eliminates x_{i-s} and
// x_{i+s} from equation i with equations i-s and i+s; after the round with
// s >= n every equation holds one unknown, x_i = d_i / b_i.  M's tridiagonal
// part is strictly diagonally dominant for alpha in (1, 2) (|w_0| + w_2 < -w_1),
// so no pivoting is needed.
// ---------------------------------------------------------------------------

// One reduction of equation i (a, b, c, d) with its neighbours at i - s (m)
// and i + s (p); has_m / has_p false outside the line.
template <typename W>
FDE_D void pcr_combine(W& a, W& b, W& c, W& d, bool has_m, W am, W bm, W cm, W dm, bool has_p, W ap, W bp, W cp,
                       W dp) {
    const W k1 = has_m ? a / bm : W(0);
    const W k2 = has_p ? c / bp : W(0);
    b = b - (has_m ? cm * k1 : W(0)) - (has_p ? ap * k2 : W(0));
    d = d - (has_m ? dm * k1 : W(0)) - (has_p ? dp * k2 : W(0));
    a = has_m ? -am * k1 : W(0);
    c = has_p ? -cp * k2 : W(0);
}

// Whole line in one CTA's shared memory (n <= kTriCtaItems * blockDim).
constexpr int kTriCtaItems = 8;

template <typename W>
FDE_NI void cta_tri_1d(const Inst& I, const Wk& wk, Combo<W> u, Epi<W> epi) {
    const int n = I.n1;
    W* a = reinterpret_cast<W*>(wk.smem);
    W* b = a + n;
    W* c = b + n;
    W* d = c + n;
    const W* tri = Prec<W>::tri(I);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a[i] = __ldg(tri + i);
        b[i] = __ldg(tri + n + i);
        c[i] = __ldg(tri + 2 * n + i);
        d[i] = u.get(i, true);
    }
    __syncthreads();
    for (int s = 1; s < n; s <<= 1) {
        W ra[kTriCtaItems], rb[kTriCtaItems], rc[kTriCtaItems], rd[kTriCtaItems];
#pragma unroll
        for (int e = 0; e < kTriCtaItems; ++e) {
            const int i = threadIdx.x + e * blockDim.x;
            if (i < n) {
                ra[e] = a[i];
                rb[e] = b[i];
                rc[e] = c[i];
                rd[e] = d[i];
                const int im = i - s, ip = i + s;
                const bool hm = im >= 0, hp = ip < n;
                const int jm = hm ? im : i, jp = hp ? ip : i;
                pcr_combine(ra[e], rb[e], rc[e], rd[e], hm, a[jm], b[jm], c[jm], d[jm], hp, a[jp], b[jp], c[jp],
                            d[jp]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kTriCtaItems; ++e) {
            const int i = threadIdx.x + e * blockDim.x;
            if (i < n) {
                a[i] = ra[e];
                b[i] = rb[e];
                c[i] = rc[e];
                d[i] = rd[e];
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) epi(i, d[i] / b[i], W(0));
    __syncthreads();
}

// A line spread over a team: the four coefficient vectors of the current
// round in one half of I.trisc, the next round's in the other, a team barrier
// per round (the neighbours at distance s belong to other CTAs).
template <typename W>
FDE_NI bool team_tri_1d(const Team& t, const Inst& I, Combo<W> u, Epi<W> epi) {
    const long long n = I.N;
    W* A = reinterpret_cast<W*>(I.trisc);
    W* B = A + 4 * n;
    const W* tri = Prec<W>::tri(I);
    long long lo, hi;
    team_range(t, n, lo, hi);
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        A[i] = __ldg(tri + i);
        A[n + i] = __ldg(tri + n + i);
        A[2 * n + i] = __ldg(tri + 2 * n + i);
        A[3 * n + i] = u.get(i, true);
    }
    if (!team_sync(t)) return false;
    for (long long s = 1; s < n; s <<= 1) {
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            W a = ldw(A + i), b = ldw(A + n + i), c = ldw(A + 2 * n + i), d = ldw(A + 3 * n + i);
            const long long im = i - s, ip = i + s;
            const bool hm = im >= 0, hp = ip < n;
            const long long jm = hm ? im : i, jp = hp ? ip : i;
            pcr_combine(a, b, c, d, hm, ldw(A + jm), ldw(A + n + jm), ldw(A + 2 * n + jm), ldw(A + 3 * n + jm), hp,
                        ldw(A + jp), ldw(A + n + jp), ldw(A + 2 * n + jp), ldw(A + 3 * n + jp));
            B[i] = a;
            B[n + i] = b;
            B[2 * n + i] = c;
            B[3 * n + i] = d;
        }
        if (!team_sync(t)) return false;
        W* tmp = A;
        A = B;
        B = tmp;
    }
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) epi(i, ldw(A + 3 * n + i) / ldw(A + n + i), W(0));
    return true;
}

// ---------------------------------------------------------------------------
// 1D, line split across a team: Np = P1 * P2, m = P2 m1 + m2, j = j1 + P1 j2.
// Column units hold cc consecutive columns m2; row units hold rows
// {j1, P1 - j1} whose spectral pairs (j, Np - j) meet in one unit.
// ---------------------------------------------------------------------------

// Columns per unit: ceil(P2 / team size), so every CTA of the team takes one
// unit when shared memory allows; the last unit may be narrower (split_width).
// A power-of-two width left up to a third of a team idle in the column phases
// whenever the team size did not divide P2 (93 CTAs on 256 columns: 64 units
// of 4), and those phases run at the FP64 rate of the busiest CTA.
template <typename W>
FDE_D int split_cols_per_unit(const AxisData& A, int team_size, int bytes) {
    const int cap = max_lines<W>(A.P1, 2, bytes);
    int cc = (A.P2 + team_size - 1) / team_size;
    if (cc > cap) cc = cap;
    if (cc > A.P2) cc = A.P2;
    return cc < 1 ? 1 : cc;
}

FDE_D int split_units(const AxisData& A, int cc) { return (A.P2 + cc - 1) / cc; }
// Columns of the unit that starts at column m2b.
FDE_D int split_width(const AxisData& A, int m2b, int cc) { return A.P2 - m2b < cc ? A.P2 - m2b : cc; }

// Element positions p (0-based) whose outputs a column unit [m2b, m2b+cc)
// produces: k = 2m, 2m+1 (1 <= k <= n), m = P2 m1 + m2, m1 < P1/2.
template <typename F>
FDE_D void split_unit_elements(const AxisData& A, int m2b, int cc, F f) {
    const int total = (A.P1 / 2) * cc * 2;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int m1 = idx / (2 * cc);
        const int rem = idx - m1 * 2 * cc;
        const long long k = 2LL * (A.P2 * m1 + m2b + (rem >> 1)) + (rem & 1);
        if (k >= 1 && k <= A.n) f(k - 1);
    }
}

// Forward column phase: pack the extension of u, P1-point FFTs, twiddle,
// Y[j1][m2].
template <typename W, int EXT>
FDE_NI void split_fwd_cols(const Team& t, const Inst& I, const Wk& wk, Combo<W> u, cx<W>* Y, int cc) {
    const AxisData& A = I.ax[0];
    const int n = A.n, Np = A.Np, P1 = A.P1, P2 = A.P2;
    cx<W>* buf = reinterpret_cast<cx<W>*>(wk.smem);
    const int tsh = wk.tw.logTW - A.logNp;
    const cx<W>* g = tw_global_table<W>(wk.tw);
    auto get = [&](int k, bool d) { return u.get(k - 1, d); };
    const int units = split_units(A, cc);
    for (int un = t.rank; un < units; un += t.size) {
        const int m2b = un * cc;
        const int wu = split_width(A, m2b, cc);
        for (int idx = threadIdx.x; idx < wu * P1; idx += blockDim.x) {
            const int c = idx % wu, m1 = idx / wu;
            buf[pad(c * P1 + m1)] = pack_elem<W, EXT>(get, P2 * m1 + m2b + c, n, Np);
        }
        __syncthreads();
        trace_mark(t, 50);
        fft_lines<W, false>(grp_cta(), buf, A.logP1, wu, P1, wk.tw);
        trace_mark(t, 51);
        for (int idx = threadIdx.x; idx < wu * P1; idx += blockDim.x) {
            const int c = idx % wu, j1 = idx / wu;
            const int m2 = m2b + c;
            Y[(long long)j1 * P2 + m2] = buf[pad(c * P1 + j1)] * g[(j1 * m2) << tsh];
        }
        __syncthreads();
        trace_mark(t, 52);
    }
}

// Row phase: P2-point FFTs of rows {j1, P1-j1}, spectral step on the pairs
// (j, Np-j), inverse FFTs, inverse twiddle; back to Y (and Y2).
//
// A CTA takes all of its row units (u = rank, rank + size, ...) in one batch
// when shared memory allows: one load, one forward FFT call over every line,
// one spectral step, one inverse call, one store.  A unit's 256-point lines
// keep one or two warps busy, so unit after unit left the phase bound by the
// latency of short FP64 dependency chains; the batch puts all of them in
// flight together.  Slot b of a batch holds lines 2b, 2b+1 (the second unused
// for units 0 and 1, which have one row) and, for two outputs, lines
// 2B + 2b, 2B + 2b + 1.
FDE_D void split_row_unit(int u, int P1, int rows[2], int& nrows) {
    nrows = u < 2 ? 1 : 2;
    rows[0] = u == 0 ? 0 : (u == 1 ? P1 / 2 : u - 1);
    rows[1] = P1 - rows[0];
}

template <typename W>
FDE_NI void split_rows(const Team& t, const Inst& I, const Wk& wk, const Mult<W> mu, cx<W>* Y, cx<W>* Y2) {
    trace_mark(t, 40);
    const AxisData& A = I.ax[0];
    const int P1 = A.P1, P2 = A.P2;
    const int tsh = wk.tw.logTW - A.logNp;
    const cx<W>* g = tw_global_table<W>(wk.tw);
    const bool two = mu.kind == kMulLam2;
    cx<W>* buf = reinterpret_cast<cx<W>*>(wk.smem);
    const int units = P1 / 2 + 1;
    const int mine = t.rank < units ? (units - 1 - t.rank) / t.size + 1 : 0;
    int per = max_lines<W>(P2, 4, wk.bytes);      // units per batch: four lines each
    if (per < 1) per = 1;
    for (int b0 = 0; b0 < mine; b0 += per) {
        const int B = mine - b0 < per ? mine - b0 : per;
        const int o2 = 2 * B * P2;                  // second output set
        for (int idx = threadIdx.x; idx < 2 * B * P2; idx += blockDim.x) {
            const int l = idx / P2, j2 = idx - l * P2;
            const int b = l >> 1, sl = l & 1;
            int rows[2], nrows;
            split_row_unit(t.rank + (b0 + b) * t.size, P1, rows, nrows);
            buf[pad(idx)] = sl < nrows ? ldw(Y + (long long)rows[sl] * P2 + j2) : mk(W(0), W(0));
        }
        __syncthreads();
        trace_mark(t, 41);
        fft_lines<W, false>(grp_cta(), buf, A.logP2, 2 * B, P2, wk.tw);
        trace_mark(t, 42);
        for (int idx = threadIdx.x; idx < B * P2; idx += blockDim.x) {
            const int b = idx / P2, q = idx - b * P2;
            const int u = t.rank + (b0 + b) * t.size;
            const int npairs = u == 0 ? P2 / 2 + 1 : (u == 1 ? P2 / 2 : P2);
            if (q >= npairs) continue;
            int rows[2], nrows;
            split_row_unit(u, P1, rows, nrows);
            const int j2 = q;
            const int sm = u >= 2 ? 1 : 0;
            const int j2m = u == 0 ? ((P2 - q) & (P2 - 1)) : P2 - 1 - q;
            const int j = rows[0] + P1 * j2;           // frequency of the first element
            const cx<W> wj = tw_L<W>(wk.tw, j, A.logNp + 1);
            const int base = 2 * b * P2;
            const int ia = base + j2, ib = base + sm * P2 + j2m;
            cx<W> a, bb, al, be, al2, be2;
            unpack_pair(buf[pad(ia)], buf[pad(ib)], wj, a, bb);
            mu.apply(j, 0, a, bb, al, be, al2, be2);
            cx<W> Qj, Qm;
            repack_pair(al, be, wj, Qj, Qm);
            buf[pad(ia)] = Qj;
            if (ib != ia) buf[pad(ib)] = Qm;
            if (two) {
                repack_pair(al2, be2, wj, Qj, Qm);
                buf[pad(o2 + ia)] = Qj;
                if (ib != ia) buf[pad(o2 + ib)] = Qm;
            }
        }
        __syncthreads();
        trace_mark(t, 43);
        fft_lines<W, true>(grp_cta(), buf, A.logP2, two ? 4 * B : 2 * B, P2, wk.tw);
        trace_mark(t, 44);
        for (int idx = threadIdx.x; idx < 2 * B * P2; idx += blockDim.x) {
            const int l = idx / P2, m2 = idx - l * P2;
            const int b = l >> 1, sl = l & 1;
            int rows[2], nrows;
            split_row_unit(t.rank + (b0 + b) * t.size, P1, rows, nrows);
            if (sl >= nrows) continue;
            const cx<W> w = conj(g[(rows[sl] * m2) << tsh]);
            Y[(long long)rows[sl] * P2 + m2] = buf[pad(idx)] * w;
            if (two) Y2[(long long)rows[sl] * P2 + m2] = buf[pad(o2 + idx)] * w;
        }
        __syncthreads();
    }
}

// Inverse column transform of one unit of cc columns (its own width) into the
// buffer (both sets when two).
template <typename W>
FDE_D void split_inv_unit_fft(const Inst& I, const Wk& wk, const cx<W>* Y, const cx<W>* Y2, int m2b, int cc,
                              bool two) {
    const AxisData& A = I.ax[0];
    const int P1 = A.P1, P2 = A.P2;
    cx<W>* buf = reinterpret_cast<cx<W>*>(wk.smem);
    for (int idx = threadIdx.x; idx < cc * P1; idx += blockDim.x) {
        const int c = idx % cc, j1 = idx / cc;
        buf[pad(c * P1 + j1)] = ldw(Y + (long long)j1 * P2 + m2b + c);
        if (two) buf[pad((cc + c) * P1 + j1)] = ldw(Y2 + (long long)j1 * P2 + m2b + c);
    }
    __syncthreads();
    fft_lines<W, true>(grp_cta(), buf, A.logP1, two ? 2 * cc : cc, P1, wk.tw);
}

// Inverse column phase: a_k (and b_k) of each unit's columns to the epilogue.
template <typename W>
FDE_NI void split_inv_cols(const Team& t, const Inst& I, const Wk& wk, const cx<W>* Y, const cx<W>* Y2, int cc,
                           bool two, Epi<W> epi) {
    const AxisData& A = I.ax[0];
    const cx<W>* buf = reinterpret_cast<const cx<W>*>(wk.smem);
    const int units = split_units(A, cc);
    for (int un = t.rank; un < units; un += t.size) {
        const int m2b = un * cc;
        const int wu = split_width(A, m2b, cc);
        split_inv_unit_fft<W>(I, wk, Y, Y2, m2b, wu, two);
        trace_mark(t, 57);
        const int total = (A.P1 / 2) * wu * 2;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int m1 = idx / (2 * wu);
            const int rem = idx - m1 * 2 * wu;
            const int c = rem >> 1, e = rem & 1;
            const long long k = 2LL * (A.P2 * m1 + m2b + c) + e;
            if (k >= 1 && k <= A.n) {
                const cx<W> q = buf[pad(c * A.P1 + m1)];
                W vb = W(0);
                if (two) {
                    const cx<W> q2 = buf[pad((wu + c) * A.P1 + m1)];
                    vb = e ? q2.y : q2.x;
                }
                epi(k - 1, e ? q.y : q.x, vb);
            }
        }
        __syncthreads();
    }
}

// tau inverse columns -> z (written to zout) -> matvec forward columns on the
// same units: the zero-padded packing of z at m = P2 m1 + m2 takes exactly
// the tau outputs k = 2m, 2m+1 of column m2.
template <typename W>
FDE_NI void split_tau_inv_mv_fwd(const Team& t, const Inst& I, const Wk& wk, const cx<W>* Yt, cx<W>* Ym, int cc,
                                 W* zout) {
    const AxisData& A = I.ax[0];
    const int P1 = A.P1, P2 = A.P2, n = A.n;
    cx<W>* buf = reinterpret_cast<cx<W>*>(wk.smem);
    const W* dinv = Prec<W>::dinv(I);
    const bool post = I.has_D && I.order == FDE_ORDER_TAU_D;
    const int units = split_units(A, cc);
    const int tsh = wk.tw.logTW - A.logNp;
    const cx<W>* g = tw_global_table<W>(wk.tw);
    for (int un = t.rank; un < units; un += t.size) {
        const int m2b = un * cc;
        const int wu = split_width(A, m2b, cc);
        split_inv_unit_fft<W>(I, wk, Yt, nullptr, m2b, wu, false);
        trace_mark(t, 53);
        for (int idx = threadIdx.x; idx < wu * P1; idx += blockDim.x) {
            const int c = idx / P1, m1 = idx - c * P1;
            const long long m = (long long)P2 * m1 + m2b + c;
            const cx<W> q = buf[pad(idx)];
            W zr[2] = {W(0), W(0)};
            if (m1 < P1 / 2) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const long long k = 2 * m + e;
                    if (k >= 1 && k <= n) {
                        W v = e ? q.y : q.x;
                        if (post) v *= __ldg(dinv + (k - 1));
                        zout[k - 1] = v;
                        zr[e] = v;
                    }
                }
            }
            buf[pad(idx)] = mk(zr[0], zr[1]);
        }
        __syncthreads();
        trace_mark(t, 54);
        fft_lines<W, false>(grp_cta(), buf, A.logP1, wu, P1, wk.tw);
        trace_mark(t, 55);
        for (int idx = threadIdx.x; idx < wu * P1; idx += blockDim.x) {
            const int c = idx % wu, j1 = idx / wu;
            const int m2 = m2b + c;
            Ym[(long long)j1 * P2 + m2] = buf[pad(c * P1 + j1)] * g[(j1 * m2) << tsh];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 2D plane: rows (x lines, contiguous) and columns (y lines, stride n1)
// ---------------------------------------------------------------------------

template <typename W>
FDE_HD int plane_lines_per_unit(int Np, int nbuf, int nlines_total, int workers, int bytes, int extra_real) {
    const int cap = max_lines<W>(Np, nbuf, bytes, extra_real);
    const int want = (nlines_total + workers - 1) / workers;
    int b = want < cap ? want : cap;
    return b < 1 ? 1 : b;
}

// Work area of one of ng groups (256-byte aligned).
FDE_HD int plane_group_bytes(int bytes, int ng) { return (bytes / ng) & ~255; }

// Thread groups per CTA of a plane phase: the two halves when a line with
// its buffers fits half the work area and the FFT's widest pass fits half
// the threads (FP32 lines up to 4096 points), else the whole CTA.  While one
// half waits on the global loads of a pack or an epilogue, the other can run
// its FFT passes.  Measured on the 4095^2 FP32 plane: the row phase that
// fuses the second sine transform with the x part of the matvec takes 6 %
// less time, the other row phases the same.
template <typename W>
FDE_HD int plane_groups(int Np, int nbuf, int bytes, int extra_real, int threads) {
    if (fft_lines_per_call(ilog2(Np), threads / 2, (int)sizeof(W)) < 1) return 1;
    return max_lines<W>(Np, nbuf, plane_group_bytes(bytes, 2), extra_real) >= 1 ? 2 : 1;
}

// Split of a plane phase over the team: units of B lines; unit un belongs to
// CTA un mod t.size (as for ng = 1, so a CTA owns the same lines whatever its
// grouping) and, in that CTA, to group (un / t.size) mod ng.
struct PlaneSplit {
    Grp g;
    unsigned char* smem;    // the group's work area
    int ng, B, units, first, step;
};

// Row phases split the CTA; column phases keep it whole, since a column unit
// of C lines reads C adjacent elements of every row, and halving C halves the
// useful bytes of every 32-byte sector loaded.
constexpr bool kRowHalves = true;
constexpr bool kColHalves = false;

template <typename W>
FDE_D PlaneSplit plane_split(const Team& t, const Wk& wk, int Np, int nbuf, int nlines, int extra_real,
                             bool halves) {
    PlaneSplit ps;
    ps.ng = halves ? plane_groups<W>(Np, nbuf, wk.bytes, extra_real, (int)blockDim.x) : 1;
    const int gi = ps.ng == 2 && (int)threadIdx.x >= (int)blockDim.x / 2 ? 1 : 0;
    ps.g = ps.ng == 2 ? grp_half(gi) : grp_cta();
    const int gb = plane_group_bytes(wk.bytes, ps.ng);
    ps.smem = wk.smem + (size_t)gi * gb;
    ps.B = plane_lines_per_unit<W>(Np, nbuf, nlines, t.size * ps.ng, gb, extra_real);
    ps.units = (nlines + ps.B - 1) / ps.B;
    ps.first = t.rank + gi * t.size;
    ps.step = ps.ng * t.size;
    return ps;
}

// Rows row0 .. row0 + nb - 1 of a plane (pitch n1, flat origin o0 = row0 n1)
// from the sine sums in sv (line l at l Np, entry p + 1): out[o] = sv (*
// post[o]), written back to sv too when BACK.  Every thread loads the post
// factors of kPackUnroll elements before any store (a store could alias
// post, so the compiler would not hoist the next load above it).
template <typename W, bool BACK>
FDE_D void rows_from_sv(const Grp& g, W* sv, int nb, int n1, int Np, long long o0, const W* post, W* out) {
    constexpr int U = kPackUnroll<W>;
    const int total = nb * n1;
    const int nt = g.nt;
    for (int base = g.tid; base < total; base += U * nt) {
        W f[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * nt;
            f[u] = (post != nullptr && idx < total) ? __ldg(post + o0 + idx) : W(1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * nt;
            if (idx < total) {
                const int l = idx / n1, p = idx - l * n1;
                const W v = sv[l * Np + p + 1] * f[u];
                if (BACK) sv[l * Np + p + 1] = v;
                out[o0 + idx] = v;
            }
        }
    }
}

// Lone DST-I along rows: out[row, j-1] = s_j (* post) of the rows of u.
template <typename W>
FDE_NI void plane_dst_rows(const Team& t, const Inst& I, const Wk& wk, Combo<W> u, const W* post, W* out) {
    const AxisData& A = I.ax[0];
    const int n1 = A.n, Np = A.Np, n2 = I.n2;
    const PlaneSplit ps = plane_split<W>(t, wk, Np, 1, n2, 1, kRowHalves);
    const Grp& g = ps.g;
    const int B = ps.B;
    cx<W>* buf = reinterpret_cast<cx<W>*>(ps.smem);
    W* sv = reinterpret_cast<W*>(buf + padded_len(B * Np));
    for (int un = ps.first; un < ps.units; un += ps.step) {
        const int row0 = un * B;
        const int nb = (n2 - row0) < B ? (n2 - row0) : B;
        cta_pack<W, kExtOdd, false>(g, buf, nb, n1, Np, [&](int l, int k, bool d) {
            return u.get((long long)(row0 + l) * n1 + (k - 1), d);
        });
        trace_mark(t, 70);
        fft_dst_lines<W>(g, buf, sv, nb, Np, A.logNp, wk.tw);
        trace_mark(t, 87);
        rows_from_sv<W, false>(g, sv, nb, n1, Np, (long long)row0 * n1, post, out);
        grp_sync(g);
    }
    __syncthreads();
}

// tau^{-1} along columns in place: z[:, c] <- S2 diag(phi) S2 z[:, c].
template <typename W>
FDE_NI void plane_tau_cols(const Team& t, const Inst& I, const Wk& wk, W* z) {
    const AxisData& A = I.ax[1];
    const int n2 = A.n, Np = A.Np, n1 = I.n1;
    const PlaneSplit ps = plane_split<W>(t, wk, Np, 1, n1, 0, kColHalves);
    const Grp& g = ps.g;
    const int C = ps.B;
    cx<W>* buf = reinterpret_cast<cx<W>*>(ps.smem);
    const Mult<W>& mu = mult_slot<W>(mult_tau2<W>(I));
    for (int un = ps.first; un < ps.units; un += ps.step) {
        const int c0 = un * C;
        const int nc = (n1 - c0) < C ? (n1 - c0) : C;
        cta_pack<W, kExtOdd, true>(g, buf, nc, n2, Np, [&](int l, int k, bool) {
            return ldw(z + (long long)(k - 1) * n1 + c0 + l);
        });
        trace_mark(t, 72);
        fft_spectral_lines<W>(g, buf, nc, Np, A.logNp, wk.tw, mu, c0, nc);
        trace_mark(t, 82);
        cta_unpack<W, true, false>(g, buf, nc, n2, Np, [&](int l, int p, W va, W) {
            z[(long long)p * n1 + c0 + l] = va;
        });
        grp_sync(g);
    }
    __syncthreads();
}

// x part of the matvec on the rows of s x; epi(o, a, b).
template <typename W>
FDE_NI void plane_matvec_rows(const Team& t, const Inst& I, const Wk& wk, const W* x, W s, Epi<W> epi) {
    const AxisData& A = I.ax[0];
    const int n1 = A.n, Np = A.Np, n2 = I.n2;
    const bool sym = I.symx;
    const PlaneSplit ps = plane_split<W>(t, wk, Np, sym ? 1 : 2, n2, 0, kRowHalves);
    const Grp& g = ps.g;
    const int B = ps.B;
    cx<W>* buf = reinterpret_cast<cx<W>*>(ps.smem);
    const Mult<W>& mu = mult_slot<W>(mult_matvec<W>(A, sym));
    for (int un = ps.first; un < ps.units; un += ps.step) {
        const int row0 = un * B;
        const int nb = (n2 - row0) < B ? (n2 - row0) : B;
        cta_pack<W, kExtZero, false>(g, buf, nb, n1, Np, [&](int l, int k, bool) {
            return s * ldw(x + (long long)(row0 + l) * n1 + (k - 1));
        });
        fft_spectral_lines<W>(g, buf, nb, Np, A.logNp, wk.tw, mu, 0, sym ? nb : 2 * nb);
        auto fe = [&](int l, int p) { return epi.fetch((long long)(row0 + l) * n1 + p); };
        auto pu = [&](int l, int p, W va, W vb, const typename Epi<W>::Ops& r) {
            epi.put((long long)(row0 + l) * n1 + p, va, vb, r);
        };
        if (sym) cta_unpack2<W, false, false>(g, buf, nb, n1, Np, fe, pu);
        else cta_unpack2<W, false, true>(g, buf, nb, n1, Np, fe, pu);
        grp_sync(g);
    }
    __syncthreads();
}

// The second sine transform of the 2D tau solve (rows of tprime, D^{-1}
// after it per the order) fused with the x part of the matvec on the same
// rows: z is written (the y part needs it) and tmp = c0 z + D_+ T z + D_- T^T z.
template <typename W>
FDE_NI void plane_dst_matvec_rows(const Team& t, const Inst& I, const Wk& wk, const W* tprime, W* z, W* tmp) {
    const AxisData& A = I.ax[0];
    const int n1 = A.n, Np = A.Np, n2 = I.n2;
    const bool sym = I.symx;
    const int nbuf = sym ? 1 : 2;
    const PlaneSplit ps = plane_split<W>(t, wk, Np, nbuf, n2, 1, kRowHalves);
    const Grp& g = ps.g;
    const int B = ps.B;
    cx<W>* buf = reinterpret_cast<cx<W>*>(ps.smem);
    W* sv = reinterpret_cast<W*>(buf + padded_len(nbuf * B * Np));
    const W* dinv = Prec<W>::dinv(I);
    const bool post = I.has_D && I.order == FDE_ORDER_TAU_D;
    const Mult<W>& mu = mult_slot<W>(mult_matvec<W>(A, sym));
    const W c0 = W(I.c0);
    const W* dp = Prec<W>::dp(I);
    const W* dm = Prec<W>::dm(I);
    for (int un = ps.first; un < ps.units; un += ps.step) {
        const int row0 = un * B;
        const int nb = (n2 - row0) < B ? (n2 - row0) : B;
        cta_pack<W, kExtOdd, false>(g, buf, nb, n1, Np, [&](int l, int k, bool) {
            return ldw(tprime + (long long)(row0 + l) * n1 + (k - 1));
        });
        trace_mark(t, 74);
        fft_dst_lines<W>(g, buf, sv, nb, Np, A.logNp, wk.tw);
        trace_mark(t, 91);
        rows_from_sv<W, true>(g, sv, nb, n1, Np, (long long)row0 * n1, post ? dinv : nullptr, z);
        grp_sync(g);
        trace_mark(t, 92);
        cta_pack<W, kExtZero, false>(g, buf, nb, n1, Np, [&](int l, int k, bool) { return sv[l * Np + k]; });
        trace_mark(t, 93);
        fft_spectral_lines<W>(g, buf, nb, Np, A.logNp, wk.tw, mu, 0, nbuf * nb);
        trace_mark(t, 96);
        auto fe = [&](int l, int p) {
            const long long o = (long long)(row0 + l) * n1 + p;
            return cx<W>{coef(dp, I.dpc, o), sym ? W(0) : coef(dm, I.dmc, o)};
        };
        auto pu = [&](int l, int p, W va, W vb, const cx<W>& d) {
            const long long o = (long long)(row0 + l) * n1 + p;
            W v = c0 * sv[l * Np + p + 1] + d.x * va;
            if (!sym) v += d.y * vb;
            tmp[o] = v;
        };
        if (sym) cta_unpack2<W, false, false>(g, buf, nb, n1, Np, fe, pu);
        else cta_unpack2<W, false, true>(g, buf, nb, n1, Np, fe, pu);
        grp_sync(g);
    }
    __syncthreads();
}

// y part: epi(o, a, b) with a, b the T_b and T_b^T (or symmetric) products
// of the columns of s x.  Column units of C columns; a CTA owns its units'
// columns.
template <typename W>
FDE_NI void plane_matvec_cols(const Team& t, const Inst& I, const Wk& wk, const W* x, W s, Epi<W> epi) {
    const AxisData& A = I.ax[1];
    const int n2 = A.n, Np = A.Np, n1 = I.n1;
    const bool sym = I.symy;
    const PlaneSplit ps = plane_split<W>(t, wk, Np, sym ? 1 : 2, n1, 0, kColHalves);
    const Grp& g = ps.g;
    const int C = ps.B;
    cx<W>* buf = reinterpret_cast<cx<W>*>(ps.smem);
    const Mult<W>& mu = mult_slot<W>(mult_matvec<W>(A, sym));
    for (int un = ps.first; un < ps.units; un += ps.step) {
        const int c0 = un * C;
        const int nc = (n1 - c0) < C ? (n1 - c0) : C;
        cta_pack<W, kExtZero, true>(g, buf, nc, n2, Np, [&](int l, int k, bool) {
            return s * ldw(x + (long long)(k - 1) * n1 + c0 + l);
        });
        trace_mark(t, 76);
        fft_spectral_lines<W>(g, buf, nc, Np, A.logNp, wk.tw, mu, 0, sym ? nc : 2 * nc);
        trace_mark(t, 85);
        auto fe = [&](int l, int p) { return epi.fetch((long long)p * n1 + c0 + l); };
        auto pu = [&](int l, int p, W va, W vb, const typename Epi<W>::Ops& r) {
            epi.put((long long)p * n1 + c0 + l, va, vb, r);
        };
        if (sym) cta_unpack2<W, true, false>(g, buf, nc, n2, Np, fe, pu);
        else cta_unpack2<W, true, true>(g, buf, nc, n2, Np, fe, pu);
        grp_sync(g);
    }
    __syncthreads();
}


// The column phases: whole column lines per CTA.
template <typename W>
FDE_D bool plane_cols_tau(const Team& t, const Inst& I, const Wk& wk, W* z) {
    plane_tau_cols<W>(t, I, wk, z);
    return true;
}

template <typename W>
FDE_D bool plane_cols_matvec(const Team& t, const Inst& I, const Wk& wk, const W* x, W s, Epi<W> epi) {
    plane_matvec_cols<W>(t, I, wk, x, s, epi);
    return true;
}

// ---------------------------------------------------------------------------
// Operators (team barrier at the end)
// ---------------------------------------------------------------------------

// y = M (s x), written per `o`.  `tmp`: N-vector of scratch (2D only).
template <typename W>
FDE_D bool op_matvec_out(const Team& t, const Inst& I, int line_mode, const W* x, W s, W* tmp, OutSpec<W> o,
                         const Wk& wk) {
    trace_mark(t, 10);
    if (I.dim == 1) {
        const Epi<W> e = epi_mvx<W>(I, x, s, o);
        if (line_mode == kLineCta) {
            if (t.rank == 0) cta_matvec_1d<W>(I, wk, x, s, e);
        } else {
            const AxisData& A = I.ax[0];
            cx<W>* Y = Prec<W>::split(I);
            const int cc = split_cols_per_unit<W>(A, t.size, wk.bytes);
            split_fwd_cols<W, kExtZero>(t, I, wk, combo_vec<W>(x, s), Y, cc);
            if (!team_sync(t)) return false;
            trace_mark(t, 11);
            split_rows<W>(t, I, wk, mult_matvec<W>(A, I.symx), Y, Y + A.Np);
            if (!team_sync(t)) return false;
            trace_mark(t, 12);
            split_inv_cols<W>(t, I, wk, Y, Y + A.Np, cc, !I.symx, e);
        }
    } else {
        plane_matvec_rows<W>(t, I, wk, x, s, epi_mvx<W>(I, x, s, out_store<W>(tmp)));
        if (!team_sync(t)) return false;
        trace_mark(t, 11);
        if (!plane_cols_matvec<W>(t, I, wk, x, s, epi_mvy<W>(I, tmp, o))) return false;
    }
    const bool ok = team_sync(t);
    trace_mark(t, 13);
    return ok;
}

template <typename W>
FDE_D bool op_matvec(const Team& t, const Inst& I, int line_mode, const W* x, W s, W* y, W* tmp, const Wk& wk) {
    return op_matvec_out<W>(t, I, line_mode, x, s, tmp, out_store<W>(y), wk);
}

// z = P^{-1} u, u given by a Combo; written per `o`.  `zbuf`: an N-vector the
// 2D path uses in place (it may be o.out).
template <typename W>
FDE_D bool op_tau_combo(const Team& t, const Inst& I, int line_mode, Combo<W> u, W* zbuf, OutSpec<W> o,
                        const Wk& wk) {
    trace_mark(t, 20);
    if (I.order == FDE_ORDER_TRI) {
        if (line_mode == kLineCta) {
            if (t.rank == 0) cta_tri_1d<W>(I, wk, u, epi_a<W>(nullptr, o));
        } else if (!team_tri_1d<W>(t, I, u, epi_a<W>(nullptr, o))) {
            return false;
        }
        const bool ok = team_sync(t);
        trace_mark(t, 23);
        return ok;
    }
    const W* dinv = Prec<W>::dinv(I);
    const bool pre = I.has_D && I.order == FDE_ORDER_D_TAU;
    const bool post = I.has_D && I.order == FDE_ORDER_TAU_D;
    if (I.dim == 1) {
        if (line_mode == kLineCta) {
            if (t.rank == 0) cta_tau_1d<W>(I, wk, u, epi_a<W>(nullptr, o));
        } else {
            const AxisData& A = I.ax[0];
            cx<W>* Y = Prec<W>::split(I);
            if (pre) u.pre = dinv;
            const int cc = split_cols_per_unit<W>(A, t.size, wk.bytes);
            split_fwd_cols<W, kExtOdd>(t, I, wk, u, Y, cc);
            if (!team_sync(t)) return false;
            trace_mark(t, 21);
            split_rows<W>(t, I, wk, mult_tau1<W>(A), Y, nullptr);
            if (!team_sync(t)) return false;
            trace_mark(t, 22);
            split_inv_cols<W>(t, I, wk, Y, nullptr, cc, false, epi_a<W>(post ? dinv : nullptr, o));
        }
    } else {
        if (pre) u.pre = dinv;
        plane_dst_rows<W>(t, I, wk, u, nullptr, zbuf);
        if (!team_sync(t)) return false;
        trace_mark(t, 21);
        if (!plane_cols_tau<W>(t, I, wk, zbuf)) return false;
        if (!team_sync(t)) return false;
        trace_mark(t, 22);
        // last sine transform along rows; a row belongs to one CTA, so reading
        // zbuf and writing the output (possibly zbuf) is safe
        if (o.outk == kOutStore) {
            plane_dst_rows<W>(t, I, wk, combo_vec<W>(zbuf, W(1)), post ? dinv : nullptr, o.out);
        } else {
            // out += z: z first into zbuf (row-local), then the update of the same rows
            plane_dst_rows<W>(t, I, wk, combo_vec<W>(zbuf, W(1)), post ? dinv : nullptr, zbuf);
            __syncthreads();
            // the rows this CTA's groups wrote: the units of plane_dst_rows' split
            const PlaneSplit ps = plane_split<W>(t, wk, I.ax[0].Np, 1, I.n2, 1, kRowHalves);
            const int B = ps.B;
            const int units = ps.units;
            const Epi<W> e = epi_a<W>(nullptr, o);
            for (int un = t.rank; un < units; un += t.size) {
                const long long o0 = (long long)un * B * I.n1;
                const long long o1 = (long long)((un + 1) * B < I.n2 ? (un + 1) * B : I.n2) * I.n1;
                for (long long p = o0 + threadIdx.x; p < o1; p += blockDim.x) e(p, ldw(zbuf + p), W(0));
            }
        }
    }
    const bool ok = team_sync(t);
    trace_mark(t, 23);
    return ok;
}

template <typename W>
FDE_D bool op_tau(const Team& t, const Inst& I, int line_mode, const W* r, W s, W* z, const Wk& wk) {
    return op_tau_combo<W>(t, I, line_mode, combo_vec(r, s), z, out_store<W>(z), wk);
}

}  // namespace fde
