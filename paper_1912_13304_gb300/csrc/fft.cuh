// Power-of-two complex FFTs for one CTA: Stockham autosort radix-8/4/2 passes
// whose butterflies run in registers.  Data sit in shared memory (in place:
// every thread stages its inputs in registers, the CTA synchronises, then
// writes) or, for the one-time symbol assembly, in global memory (ping-pong).
//
// Shared-memory line buffers are indexed through pad(i) = i + i/16: one
// spare complex every 16 keeps every Stockham read and write pattern at the
// minimum number of bank wavefronts (the radix-8 first pass writes at stride
// 8 and would otherwise be 8- to 16-way conflicted).
//
// Conventions: forward X_j = sum_k x_k w^{jk}, w = exp(-2 pi i / P); inverse
// uses w^{-1} and is unnormalised.  Radix twiddles come from a quarter-wave
// FP64 table of W_T in shared memory when P <= T, else from the global
// table of W_TW.
#pragma once

#include "common.cuh"

namespace fde {

FDE_HD int pad(int i) { return i + (i >> 4); }
FDE_HD int padded_len(int n) { return n + (n >> 4) + 1; }

// Twiddle sources of one CTA.
struct Tw {
    const cx<double>* q;       // shared memory: W_T^t for t < T/4 (quarter wave), entry t at pad(t)
    const cx<float>* q32;      // the same table rounded to FP32
    int logT;
    const cx<double>* g64;     // global: W_TW^t for t < TW
    const cx<float>* g32;
    int logTW;
};

template <typename R> FDE_D const cx<R>* tw_global_table(const Tw& t);
template <> FDE_D const cx<double>* tw_global_table<double>(const Tw& t) { return t.g64; }
template <> FDE_D const cx<float>* tw_global_table<float>(const Tw& t) { return t.g32; }

// W_T^idx (idx < T) from the quarter table: W^{q T/4 + r} = (-i)^q W^r.
template <typename R> FDE_D cx<R> tw_quarter_entry(const Tw& t, int r);
template <> FDE_D cx<double> tw_quarter_entry<double>(const Tw& t, int r) { return t.q[pad(r)]; }
template <> FDE_D cx<float> tw_quarter_entry<float>(const Tw& t, int r) { return t.q32[pad(r)]; }

// Sign flip by an integer XOR of the sign bit (flip = 0 or 1), which keeps
// the selection off the floating-point pipes.
FDE_D double flip_sign(double v, int flip) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)flip << 63));
}
FDE_D float flip_sign(float v, int flip) { return __int_as_float(__float_as_int(v) ^ (flip << 31)); }

// Branch-free: quadrants 1 and 3 swap the components, the first component is
// negated in quadrants 2 and 3, the second in quadrants 1 and 2.
template <typename R>
FDE_D cx<R> tw_quarter(const Tw& t, int idx) {
    const int q = (idx >> (t.logT - 2)) & 3;
    const int r = idx & ((1 << (t.logT - 2)) - 1);
    const cx<R> w = tw_quarter_entry<R>(t, r);
    const R a = (q & 1) ? w.y : w.x;
    const R b = (q & 1) ? w.x : w.y;
    return mk(flip_sign(a, q >> 1), flip_sign(b, ((q + 1) >> 1) & 1));
}

// W_L^j for the real-packing step (L = 2^logL, any size): global table.
template <typename R>
FDE_D cx<R> tw_L(const Tw& t, long long j, int logL) {
    return tw_global_table<R>(t)[j << (t.logTW - logL)];
}

// ---------------------------------------------------------------------------
// Register DFTs
// ---------------------------------------------------------------------------

template <typename R, bool INV>
FDE_D cx<R> rot_quarter(cx<R> a) {   // multiply by w_4 = -i (forward) or +i (inverse)
    return INV ? mul_i(a) : mul_mi(a);
}

template <typename R, bool INV>
FDE_D void dft2(cx<R>& a, cx<R>& b) {
    cx<R> t = a - b;
    a = a + b;
    b = t;
}

template <typename R, bool INV>
FDE_D void dft4(cx<R>* v) {           // v[0..3] in, natural order out
    cx<R> s0 = v[0] + v[2], d0 = v[0] - v[2];
    cx<R> s1 = v[1] + v[3], d1 = rot_quarter<R, INV>(v[1] - v[3]);
    v[0] = s0 + s1;
    v[2] = s0 - s1;
    v[1] = d0 + d1;
    v[3] = d0 - d1;
}

template <typename R, bool INV>
FDE_D void dft8(cx<R>* v) {
    cx<R> e[4] = {v[0], v[2], v[4], v[6]};
    cx<R> o[4] = {v[1], v[3], v[5], v[7]};
    dft4<R, INV>(e);
    dft4<R, INV>(o);
    const R h = R(0.70710678118654752440084436210485);
    // w_8^1 = (1 - i)/sqrt2 forward, (1 + i)/sqrt2 inverse
    cx<R> o1 = INV ? mk(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                   : mk(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    cx<R> o2 = rot_quarter<R, INV>(o[2]);
    // w_8^3 = (-1 - i)/sqrt2 forward, (-1 + i)/sqrt2 inverse
    cx<R> o3 = INV ? mk(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                   : mk(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = e[2] + o2;
    v[6] = e[2] - o2;
    v[3] = e[3] + o3;
    v[7] = e[3] - o3;
}

// a W_16^E (forward) or a W_16^-E (inverse), W_16 = exp(-2 pi i / 16), for the
// exponents that the 4 x 4 split of a 16-point DFT needs (radix16_item).
template <typename R, bool INV, int E>
FDE_D cx<R> w16(cx<R> a) {
    const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173), h = R(0.70710678118654752440);
    R wr, wi;   // W_16^E = wr - i wi
    if constexpr (E == 1) { wr = c1; wi = s1; }
    else if constexpr (E == 2) { wr = h; wi = h; }
    else if constexpr (E == 3) { wr = s1; wi = c1; }
    else if constexpr (E == 6) { wr = -h; wi = h; }
    else { wr = -c1; wi = -s1; }                    // E == 9
    if (!INV) wi = -wi;
    return mk(a.x * wr - a.y * wi, a.x * wi + a.y * wr);
}

template <typename R, int RAD, bool INV>
FDE_D void dft_reg(cx<R>* v) {
    if constexpr (RAD == 2) dft2<R, INV>(v[0], v[1]);
    else if constexpr (RAD == 4) dft4<R, INV>(v);
    else dft8<R, INV>(v);
}

// ---------------------------------------------------------------------------
// One Stockham pass over `nlines` lines of length P (= 2^logP) at stride
// `lstride` (flat, unpadded indices).  Item j of a line reads x[j + r P/RAD],
// applies the twiddles w_{Ns RAD}^{r k} (k = j mod Ns), a radix-RAD DFT, and
// writes y[(j - k) RAD + k + r Ns].
// ---------------------------------------------------------------------------

// One radix-16 item, column by column of the 4 x 4 split (r = n2 + 4 n1): the
// four inputs of column n2 are loaded, twiddled by w^(r k) and transformed
// (DFT4 over n1) before the next column's loads, so at most the 16 partial
// results, one column's inputs and the base twiddles are live (no spills in
// a kernel of 128 registers, against 19 local loads per item when the 16
// inputs were loaded first).  The twiddle powers are products of w, w^2, w^4
// and w^8 from the table, at most three roundings each.  Output X[k1 + 4 k2]
// lands in y[k1 + 4 k2].
template <typename R, bool INV>
FDE_D void radix16_item(const cx<R>* buf, int o, int logItems, int k, bool tw_on, int twsh, bool smem_tw,
                        const Tw& tw, const cx<R>* gtab, cx<R>* y) {
    auto look = [&](int e) {
        const int idx = (e * k) << twsh;
        const cx<R> w = smem_tw ? tw_quarter<R>(tw, idx) : gtab[idx];
        return INV ? conj(w) : w;
    };
    cx<R> w1 = mk(R(1), R(0)), w2 = w1, w4 = w1, w8 = w1;
    if (tw_on) { w1 = look(1); w2 = look(2); w4 = look(4); w8 = look(8); }
    const cx<R> w12 = w4 * w8;
    cx<R> c[4][4];                           // c[k1][n2]
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        cx<R> t4[4];
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) t4[n1] = buf[pad(o + ((n2 + 4 * n1) << logItems))];
        if (tw_on) {
            cx<R> wb = w1;                   // w^n2
            if (n2 == 2) wb = w2;
            if (n2 == 3) wb = w1 * w2;
            if (n2 > 0) t4[0] = t4[0] * wb;
            t4[1] = t4[1] * (n2 > 0 ? wb * w4 : w4);
            t4[2] = t4[2] * (n2 > 0 ? wb * w8 : w8);
            t4[3] = t4[3] * (n2 > 0 ? wb * w12 : w12);
        }
        dft4<R, INV>(t4);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) c[k1][n2] = t4[k1];
    }
    c[1][1] = w16<R, INV, 1>(c[1][1]);
    c[1][2] = w16<R, INV, 2>(c[1][2]);
    c[1][3] = w16<R, INV, 3>(c[1][3]);
    c[2][1] = w16<R, INV, 2>(c[2][1]);
    c[2][2] = rot_quarter<R, INV>(c[2][2]);
    c[2][3] = w16<R, INV, 6>(c[2][3]);
    c[3][1] = w16<R, INV, 3>(c[3][1]);
    c[3][2] = w16<R, INV, 6>(c[3][2]);
    c[3][3] = w16<R, INV, 9>(c[3][3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        cx<R> t4[4] = {c[k1][0], c[k1][1], c[k1][2], c[k1][3]};
        dft4<R, INV>(t4);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = t4[k2];
    }
}

template <typename R, int RAD, int EPT, bool INV>
FDE_D void stockham_pass_inplace(const Grp& g, cx<R>* buf, int logP, int nlines, int lstride, int logNs,
                                 const Tw& tw, bool smem_tw) {
    constexpr int K = EPT / RAD;                // items per thread
    constexpr int LR = RAD == 16 ? 4 : (RAD == 8 ? 3 : (RAD == 4 ? 2 : 1));
    const int logItems = logP - LR;             // items per line = P / RAD
    const int total = nlines << logItems;
    const int Ns = 1 << logNs;
    const int twsh = (smem_tw ? tw.logT : tw.logTW) - logNs - LR;
    const cx<R>* gtab = tw_global_table<R>(tw);
    cx<R> v[K][RAD];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const int it = g.tid + t * g.nt;
        if (it < total) {
            const int line = it >> logItems;
            const int j = it & ((1 << logItems) - 1);
            const int base = line * lstride;
            const int k = j & (Ns - 1);
            if constexpr (RAD == 16) {
                radix16_item<R, INV>(buf, base + j, logItems, k, Ns > 1, twsh, smem_tw, tw, gtab, v[t]);
            } else {
#pragma unroll
                for (int r = 0; r < RAD; ++r) v[t][r] = buf[pad(base + j + (r << logItems))];
                if (Ns > 1) {
#pragma unroll
                    for (int r = 1; r < RAD; ++r) {
                        const int idx = (r * k) << twsh;
                        cx<R> w = smem_tw ? tw_quarter<R>(tw, idx) : gtab[idx];
                        if (INV) w = conj(w);
                        v[t][r] = v[t][r] * w;
                    }
                }
                dft_reg<R, RAD, INV>(v[t]);
            }
        }
    }
    grp_sync(g);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const int it = g.tid + t * g.nt;
        if (it < total) {
            const int line = it >> logItems;
            const int j = it & ((1 << logItems) - 1);
            const int k = j & (Ns - 1);
            const int dst = line * lstride + (j - k) * RAD + k;
#pragma unroll
            for (int r = 0; r < RAD; ++r) buf[pad(dst + r * Ns)] = v[t][r];
        }
    }
    grp_sync(g);
}

// In-place FFT of nlines lines held in (padded) shared memory, every pass
// one radix item per thread (registers hold RAD values), so a call requires
// nlines * P / RAD <= kFftItems<R> * (threads of the group) for the smallest
// radix it uses.
//
// Radix items per thread and pass.  One: two items per thread (measured for
// FP32 with 512 threads, and for both precisions with 256 threads and twice
// the registers) raised the register saves of every phase function and was
// slower overall.
template <typename R> constexpr int kFftItems = 1;

// Radix schedule of a 2^logP-point FFT, packed: log2 of pass i's radix in
// bits [4i, 4i + 4), zero after the last pass (at most 8 passes).  A packed
// word stays in a register, where an array indexed by the pass number would
// live in local memory and cost a load at the start of every pass.  FP64
// takes radix-8 passes and one radix-4 or radix-2 remainder.  FP32 takes
// radix-16 passes (twice the work between two CTA barriers, and the
// registers to hold it) and makes the smallest radix as large as possible,
// since the widest pass bounds the lines one call can take.
FDE_HD unsigned fft_schedule(int logP, int elem_bytes) {
    unsigned s = 0;
    int n = 0;
    auto put = [&](int lr) { s |= (unsigned)lr << (4 * n++); };
    if (elem_bytes == 8) {
        int rem = logP;
        while (rem >= 3) { put(3); rem -= 3; }
        if (rem > 0) put(rem);
        return s;
    }
    const int n16 = logP / 4, r = logP % 4;
    int k16 = n16;
    if (r == 2 && n16 >= 1) k16 = n16 - 1;
    if (r == 1) k16 = n16 >= 2 ? n16 - 2 : 0;
    for (int i = 0; i < k16; ++i) put(4);
    if (r == 3) put(3);
    else if (r == 2) {
        if (n16 >= 1) { put(3); put(3); } else put(2);
    } else if (r == 1) {
        if (n16 >= 2) { put(3); put(3); put(3); }
        else if (n16 == 1) { put(3); put(2); }
        else put(1);
    }
    return s;
}

template <typename R, bool INV>
FDE_D void fft_inplace(const Grp& g, cx<R>* buf, int logP, int nlines, int lstride, const Tw& tw) {
    constexpr int K = kFftItems<R>;
    const bool smem_tw = logP <= tw.logT;
    int logNs = 0;
    for (unsigned s = fft_schedule(logP, (int)sizeof(R)); s != 0; s >>= 4) {
        const int lr = (int)(s & 15u);
        if constexpr (sizeof(R) == 4) {
            if (lr == 4) {
                stockham_pass_inplace<R, 16, 16 * K, INV>(g, buf, logP, nlines, lstride, logNs, tw, smem_tw);
                logNs += 4;
                continue;
            }
        }
        if (lr == 3) stockham_pass_inplace<R, 8, 8 * K, INV>(g, buf, logP, nlines, lstride, logNs, tw, smem_tw);
        else if (lr == 2) stockham_pass_inplace<R, 4, 4 * K, INV>(g, buf, logP, nlines, lstride, logNs, tw, smem_tw);
        else stockham_pass_inplace<R, 2, 2 * K, INV>(g, buf, logP, nlines, lstride, logNs, tw, smem_tw);
        logNs += lr;
    }
}

// Radix items per line of the widest pass (the one with the smallest radix),
// and the lines one call of fft_inplace can take.
FDE_HD int fft_items_per_line(int logP, int elem_bytes) {
    const unsigned s0 = fft_schedule(logP, elem_bytes);
    if (s0 == 0) return 1;
    int mn = 4;
    for (unsigned s = s0; s != 0; s >>= 4) mn = (int)(s & 15u) < mn ? (int)(s & 15u) : mn;
    return 1 << (logP - mn);
}
FDE_HD int fft_lines_per_call(int logP, int threads, int elem_bytes) {
    return threads * (elem_bytes == 4 ? kFftItems<float> : kFftItems<double>) / fft_items_per_line(logP, elem_bytes);
}

// FFT of nlines lines of 2^logP at stride lstride (flat index), in batches
// of lines; the flat origin of a batch starting at line l0 is pad(l0 *
// lstride), which commutes with pad() because lstride is a multiple of 16
// whenever more than one batch is needed.  A single line with more radix
// items than kFftItems<R> per thread is not supported (callers split such
// lines).
template <typename R, bool INV>
FDE_D void fft_lines_in(const Grp& g, cx<R>* buf, int logP, int nlines, int lstride, const Tw& tw) {
    const int cap = fft_lines_per_call(logP, g.nt, (int)sizeof(R));
    for (int l0 = 0; l0 < nlines; l0 += cap) {
        const int nl = (nlines - l0) < cap ? (nlines - l0) : cap;
        fft_inplace<R, INV>(g, buf + pad(l0 * lstride), logP, nl, lstride, tw);
    }
}

// The same, not inlined: the radix passes get the thread's registers, at the
// price of the register saves of a call.  Callers with a spectral step
// between two transforms use the fused calls of the line layer instead, which
// pay that price once.
template <typename R, bool INV>
FDE_NI void fft_lines(const Grp g, cx<R>* buf, int logP, int nlines, int lstride, const Tw& tw) {
    fft_lines_in<R, INV>(g, buf, logP, nlines, lstride, tw);
}

// Ping-pong variant for one long line in global memory (one CTA, symbol
// assembly only).  Returns the buffer that holds the result.
// Item j of one ping-pong Stockham pass (the same steps as the shared-memory
// pass, on global buffers).
template <typename R, int RAD, bool INV>
FDE_D void stockham_item_pp(const cx<R>* src, cx<R>* dst, int j, int logItems, int Ns, int twsh, const cx<R>* tw) {
    const int k = j & (Ns - 1);
    cx<R> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[j + (r << logItems)];
    if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
            cx<R> w = tw[(r * k) << twsh];
            if (INV) w = conj(w);
            v[r] = v[r] * w;
        }
    }
    dft_reg<R, RAD, INV>(v);
    const int d = (j - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[d + r * Ns] = v[r];
}

template <typename R, int RAD, bool INV>
FDE_D void stockham_pass_pp(const cx<R>* src, cx<R>* dst, int logP, int logNs, const cx<R>* tw,
                            int logTW) {
    constexpr int LR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
    const int logItems = logP - LR;
    const int items = 1 << logItems;
    const int Ns = 1 << logNs;
    const int twsh = logTW - logNs - LR;
    for (int j = threadIdx.x; j < items; j += blockDim.x)
        stockham_item_pp<R, RAD, INV>(src, dst, j, logItems, Ns, twsh, tw);
    __syncthreads();
}

template <typename R, bool INV>
FDE_D cx<R>* fft_pingpong(cx<R>* a, cx<R>* b, int logP, const cx<R>* tw, int logTW) {
    int logNs = 0;
    int rem = logP;
    cx<R>* src = a;
    cx<R>* dst = b;
    while (rem > 0) {
        if (rem >= 3) {
            stockham_pass_pp<R, 8, INV>(src, dst, logP, logNs, tw, logTW);
            logNs += 3;
            rem -= 3;
        } else if (rem == 2) {
            stockham_pass_pp<R, 4, INV>(src, dst, logP, logNs, tw, logTW);
            logNs += 2;
            rem -= 2;
        } else {
            stockham_pass_pp<R, 2, INV>(src, dst, logP, logNs, tw, logTW);
            logNs += 1;
            rem -= 1;
        }
        cx<R>* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

}  // namespace fde
