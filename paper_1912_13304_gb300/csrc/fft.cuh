// Power-of-two complex FFTs for one CTA: Stockham autosort radix-8/4/2 passes
// whose butterflies run in registers.  Data may sit in shared memory
// (in place: every thread stages its inputs in registers, the CTA
// synchronises, then writes) or in global memory (ping-pong between two
// buffers, used only by the one-time symbol assembly).
//
// Conventions: forward X_j = sum_k x_k w^{jk}, w = exp(-2 pi i / P); inverse
// uses w^{-1} and is unnormalised.  Twiddles come from a table
// tw[t] = exp(-2 pi i t / TW), TW a power of two >= P.
#pragma once

#include "common.cuh"

namespace fde {

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

template <typename R, int RAD, bool INV>
FDE_D void dft_reg(cx<R>* v) {
    if constexpr (RAD == 2) dft2<R, INV>(v[0], v[1]);
    else if constexpr (RAD == 4) dft4<R, INV>(v);
    else dft8<R, INV>(v);
}

template <typename R, bool INV>
FDE_D cx<R> twiddle(const cx<R>* tw, int idx) {
    cx<R> w = tw[idx];
    return INV ? conj(w) : w;
}

// ---------------------------------------------------------------------------
// One Stockham pass over `nlines` lines of length P (= 2^logP) at stride
// `lstride`.  Item j of a line reads x[j + r P/RAD], applies the twiddles
// w_{Ns RAD}^{r k} (k = j mod Ns), a radix-RAD DFT, and writes
// y[(j - k) RAD + k + r Ns].
// ---------------------------------------------------------------------------

template <typename R, int RAD, int EPT, bool INV>
FDE_D void stockham_pass_inplace(cx<R>* buf, int logP, int nlines, int lstride, int logNs,
                                 const cx<R>* tw, int logTW) {
    constexpr int K = EPT / RAD;                // items per thread
    constexpr int LR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
    const int logItems = logP - LR;             // items per line = P / RAD
    const int total = nlines << logItems;
    const int Ns = 1 << logNs;
    const int twsh = logTW - logNs - LR;        // table step for w_{Ns RAD}
    cx<R> v[K][RAD];
    int dst[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const int it = threadIdx.x + t * blockDim.x;
        dst[t] = -1;
        if (it < total) {
            const int line = it >> logItems;
            const int j = it & ((1 << logItems) - 1);
            cx<R>* base = buf + (long long)line * lstride;
            const int k = j & (Ns - 1);
#pragma unroll
            for (int r = 0; r < RAD; ++r) v[t][r] = base[j + (r << logItems)];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < RAD; ++r) v[t][r] = v[t][r] * twiddle<R, INV>(tw, (r * k) << twsh);
            }
            dft_reg<R, RAD, INV>(v[t]);
            dst[t] = line * lstride + (j - k) * RAD + k;
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < K; ++t) {
        if (dst[t] >= 0) {
#pragma unroll
            for (int r = 0; r < RAD; ++r) buf[dst[t] + r * Ns] = v[t][r];
        }
    }
    __syncthreads();
}

// In-place FFT of nlines lines held in shared memory.  Requires
// nlines * P <= EPT * blockDim.x (every element staged in registers once).
template <typename R, int EPT, bool INV>
FDE_NI void fft_inplace(cx<R>* buf, int logP, int nlines, int lstride, const cx<R>* tw, int logTW) {
    int logNs = 0;
    int rem = logP;
    while (rem >= 3) {
        stockham_pass_inplace<R, 8, EPT, INV>(buf, logP, nlines, lstride, logNs, tw, logTW);
        logNs += 3;
        rem -= 3;
    }
    if (rem == 2) stockham_pass_inplace<R, 4, EPT, INV>(buf, logP, nlines, lstride, logNs, tw, logTW);
    else if (rem == 1) stockham_pass_inplace<R, 2, EPT, INV>(buf, logP, nlines, lstride, logNs, tw, logTW);
}

// Ping-pong variant for one long line in global memory (one CTA).  Returns the
// buffer that holds the result.
template <typename R, int RAD, bool INV>
FDE_D void stockham_pass_pp(const cx<R>* src, cx<R>* dst, int logP, int logNs, const cx<R>* tw,
                            int logTW) {
    constexpr int LR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
    const int logItems = logP - LR;
    const int items = 1 << logItems;
    const int Ns = 1 << logNs;
    const int twsh = logTW - logNs - LR;
    for (int j = threadIdx.x; j < items; j += blockDim.x) {
        const int k = j & (Ns - 1);
        cx<R> v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[r] = src[j + (r << logItems)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) v[r] = v[r] * twiddle<R, INV>(tw, (r * k) << twsh);
        }
        dft_reg<R, RAD, INV>(v);
        const int d = (j - k) * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) dst[d + r * Ns] = v[r];
    }
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
