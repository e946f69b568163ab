// Host side of libfde: validation, workspace layout, symbol assembly kernels
// and the C ABI declared in include/fde.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include <cuda.h>   // CUcontext and CUresult (types only)

#include "launch.h"

using namespace fde;

struct fde_plan {
    fde_problem prob;
    fde_solve_opts opts;
    Inst inst;              // host copy of the device record
    Inst* inst_dev;
    SyncArea* sync_dev;
    void* ws;
    size_t ws_bytes;
    int device;
    int smem_bytes;
    int grid[3];            // co-resident CTAs of each engine mode
    int ctas;               // CTAs of single-plan launches (0: all co-resident)
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }
bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// ---------------------------------------------------------------------------
// Per-device engine preparation (kernel attributes and occupancy)
// ---------------------------------------------------------------------------

struct DeviceInfo {
    bool ready = false;
    int num_sms = 0;
    int smem_bytes = 0;
    int grid[3] = {0, 0, 0};
};
std::mutex g_mu;
DeviceInfo g_dev[64];

cudaError_t prepare_device(int dev, DeviceInfo** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    DeviceInfo& d = g_dev[dev];
    if (!d.ready) {
        int sms = 0, optin = 0;
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        // leave room for the kernel's static shared memory (instance record, reductions)
        int smem = optin - 4096;
        if (smem > 224 * 1024) smem = 224 * 1024;
        smem &= ~255;
        for (int mode = 0; mode < 3; ++mode) {
            KernelInfo ki{};
            e = mode == 0 ? engine_prepare_f64(smem, &ki)
                          : (mode == 1 ? engine_prepare_f32(smem, &ki) : engine_prepare_ir(smem, &ki));
            if (e != cudaSuccess) return e;
            if (ki.blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
            int g = ki.blocks_per_sm * sms;
            if (g > kMaxCtas) g = kMaxCtas;
            d.grid[mode] = g;
        }
        d.num_sms = sms;
        d.smem_bytes = smem;
        d.ready = true;
    }
    *out = &d;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Validation and derived quantities
// ---------------------------------------------------------------------------

bool valid_order(double a) { return std::isfinite(a) && a > 1.0 && a < 2.0; }

bool coeff_ok(const double* arr, double c) { return arr != nullptr || (std::isfinite(c) && c >= 0.0); }

fde_status validate(const fde_problem* p, const fde_solve_opts* o) {
    if (!p || !o) return FDE_EINVAL;
    if (p->dim != 1 && p->dim != 2) return FDE_EINVAL;
    if (p->n1 < 1 || !is_pow2((long long)p->n1 + 1) || p->n1 + 1 > (1 << 22)) return FDE_EINVAL;
    if (!valid_order(p->alpha)) return FDE_EINVAL;
    if (!(p->len1 > 0.0) || !std::isfinite(p->len1) || !(p->dt > 0.0) || !std::isfinite(p->dt)) return FDE_EINVAL;
    if (p->scheme != FDE_SCHEME_IMPLICIT_EULER && p->scheme != FDE_SCHEME_CRANK_NICOLSON) return FDE_EINVAL;
    if (p->weights != FDE_WEIGHTS_GL1 && p->weights != FDE_WEIGHTS_WSGD2) return FDE_EINVAL;
    if (p->order != FDE_ORDER_TAU_D && p->order != FDE_ORDER_D_TAU && p->order != FDE_ORDER_TAU_DF &&
        p->order != FDE_ORDER_TRI)
        return FDE_EINVAL;
    // P_F-tilde and P_tri: 1D, unshifted
    if ((p->order == FDE_ORDER_TAU_DF || p->order == FDE_ORDER_TRI) && (p->dim != 1 || p->tau_shift))
        return FDE_EINVAL;
    if (p->tau_shift != 0 && p->tau_shift != 1) return FDE_EINVAL;
    if (!coeff_ok(p->dp, p->dp_const) || !coeff_ok(p->dm, p->dm_const)) return FDE_EINVAL;
    if (p->dim == 2) {
        if (p->n2 < 1 || !is_pow2((long long)p->n2 + 1) || p->n2 + 1 > 4096) return FDE_EINVAL;
        if (p->n1 + 1 > 4096) return FDE_EINVAL;
        if (!valid_order(p->beta)) return FDE_EINVAL;
        if (!(p->len2 > 0.0) || !std::isfinite(p->len2)) return FDE_EINVAL;
        if (!coeff_ok(p->ep, p->ep_const) || !coeff_ok(p->em, p->em_const)) return FDE_EINVAL;
    }
    if (p->tau_shift) {
        // 1D: constants (Case I) or arrays (the shift c0/mean(D) beside D);
        // 2D: constants only (P_hat)
        if (p->dim == 2 && (p->dp || p->dm)) return FDE_EINVAL;
        if (!p->dp && !p->dm && !(p->dp_const + p->dm_const > 0.0)) return FDE_EINVAL;
        if (p->dim == 2 && (p->ep || p->em || !(p->ep_const + p->em_const > 0.0))) return FDE_EINVAL;
    } else {
        // D = mean of the coefficients must be invertible; arrays are checked by the caller
        if (!p->dp && !p->dm && !(p->dp_const + p->dm_const > 0.0) && p->dim == 1) return FDE_EINVAL;
    }
    if (o->method != FDE_PCG && o->method != FDE_GMRES) return FDE_EINVAL;
    if (o->method == FDE_GMRES && (o->restart < 1 || o->restart > kMaxRestart)) return FDE_EINVAL;
    if (!(o->tol > 0.0) || !std::isfinite(o->tol) || o->max_iters < 1) return FDE_EINVAL;
    if (o->precision < FDE_PREC_F64 || o->precision > FDE_PREC_F32_IR) return FDE_EINVAL;
    if (o->precision == FDE_PREC_F32_IR && (!(o->inner_tol > 0.0) || o->inner_tol >= 1.0 || o->max_outer < 1))
        return FDE_EINVAL;
    if (o->side != FDE_SIDE_RIGHT && o->side != FDE_SIDE_LEFT) return FDE_EINVAL;
    if (o->method == FDE_PCG) {
        // PCG needs a symmetric M (d_+ = d_-, e_+ = e_-) and a symmetric positive P (D constant)
        const bool symx = p->dp == p->dm && (p->dp != nullptr || p->dp_const == p->dm_const);
        const bool symy = p->dim == 1 || (p->ep == p->em && (p->ep != nullptr || p->ep_const == p->em_const));
        const bool constD = !p->dp && !p->dm && (p->dim == 1 || (!p->ep && !p->em));
        if (!symx || !symy || !constD) return FDE_EINVAL;
    }
    return FDE_OK;
}

struct Layout {
    size_t inst, sync, tw64, tw32;
    size_t lam64[2], lam32[2], phi64[2], phi32[2];
    size_t dinv64, dinv32, dp32, dm32, ep32, em32;
    size_t r64, t64, wvec, split64, split32, wts, dbar, tri64, tri32, trisc;
    size_t total;
    int TW, logTW;
    int Np[2];
    bool has_D;
};

// D^{-1} is applied unless the shifted symbol absorbs a constant D (Case I, P_hat).
bool compute_has_D(const fde_problem* p) {
    if (p->order == FDE_ORDER_TAU_DF) return false;      // D folded into the symbol
    if (p->order == FDE_ORDER_TRI) return false;         // P_tri: no D
    return !p->tau_shift || (p->dim == 1 && (p->dp || p->dm));
}

Layout layout(const fde_problem* p, const fde_solve_opts* o) {
    Layout L{};
    const long long N = (long long)p->n1 * (p->dim == 2 ? p->n2 : 1);
    L.Np[0] = p->n1 + 1;
    L.Np[1] = p->dim == 2 ? p->n2 + 1 : 1;
    const int Lmax = 2 * std::max(L.Np[0], L.Np[1]);
    L.TW = std::max(Lmax, 16);
    L.logTW = ilog2(L.TW);
    L.has_D = compute_has_D(p);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes); return at; };
    L.inst = take(sizeof(Inst));
    L.sync = take(sizeof(SyncArea));
    L.tw64 = take((size_t)L.TW * sizeof(cx<double>));
    L.tw32 = take((size_t)L.TW * sizeof(cx<float>));
    for (int a = 0; a < p->dim; ++a) {
        const size_t np1 = (size_t)L.Np[a] + 1;
        L.lam64[a] = take(np1 * sizeof(cx<double>));
        L.lam32[a] = take(np1 * sizeof(cx<float>));
        L.phi64[a] = take(np1 * sizeof(double));
        L.phi32[a] = take(np1 * sizeof(float));
    }
    L.dinv64 = L.has_D ? take(N * sizeof(double)) : 0;
    L.dinv32 = L.has_D ? take(N * sizeof(float)) : 0;
    L.dp32 = p->dp ? take(N * sizeof(float)) : 0;
    L.dm32 = p->dm ? (p->dm == p->dp ? L.dp32 : take(N * sizeof(float))) : 0;
    L.ep32 = (p->dim == 2 && p->ep) ? take(N * sizeof(float)) : 0;
    L.em32 = (p->dim == 2 && p->em) ? (p->em == p->ep ? L.ep32 : take(N * sizeof(float))) : 0;
    L.r64 = take(N * sizeof(double));
    L.t64 = take(N * sizeof(double));
    const size_t wsz = o->precision == FDE_PREC_F64 ? sizeof(double) : sizeof(float);
    const long long nvec = o->method == FDE_GMRES ? (o->restart + 4) : 5;
    const long long extra = o->precision == FDE_PREC_F64 ? 0 : 2;
    size_t wbytes = (size_t)(nvec + extra) * N * wsz;
    // refinement plans may finish a solve in FP64 (the same vectors at FP64 size)
    if (o->precision == FDE_PREC_F32_IR) wbytes = std::max<size_t>(wbytes, (size_t)nvec * (size_t)N * sizeof(double));
    L.wvec = take(wbytes);
    const int npmax = std::max(L.Np[0], L.Np[1]);
    L.split64 = take((size_t)2 * npmax * sizeof(cx<double>));
    L.split32 = take((size_t)2 * npmax * sizeof(cx<float>));
    L.wts = take((size_t)(npmax + 2) * sizeof(double));
    L.dbar = take(sizeof(double));
    if (p->order == FDE_ORDER_TRI) {
        L.tri64 = take((size_t)3 * N * sizeof(double));
        L.tri32 = take((size_t)3 * N * sizeof(float));
        L.trisc = take((size_t)8 * N * sizeof(double));
    }
    L.total = off;
    return L;
}

// ---------------------------------------------------------------------------
// Assembly kernels (FP64)
// ---------------------------------------------------------------------------

__global__ void k_twiddles(cx<double>* tw64, cx<float>* tw32, int TW) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < TW; t += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)t / (double)TW, &s, &c);
        tw64[t] = mk(c, s);
        tw32[t] = mk((float)c, (float)s);
    }
}

struct AxisJob {
    int n, Np, logNp, logTW, weights;
    double alpha;
    int kind;              // 0: 1D tau multiplier 1/(L (add + mult F)); 1: 2D axis part add + mult F
    double add, mult;
    const double* dbar;    // kind 0 with a variable D: multiplier 1/(L (F + add / dbar))
    int fold_d;            // kind 0, P_F-tilde: multiplier 1/(L D_j F_j), D_j = (d_+ + d_-)/2 at x_j
    const double *dp, *dm;
    double dpc, dmc;
    const cx<double>* tw64;
    cx<double>* lam64;
    cx<float>* lam32;
    double* phi64;
    float* phi32;
    double* wts;
    cx<double>* bufA;
    cx<double>* bufB;
};

// F_alpha(theta_j), theta_j = j pi / Np: p_alpha (first order) or q_alpha
// (WSGD).  With 1 - e^{i t} = 2 sin(t/2) e^{i (t - pi)/2}:
//   p = -2 rho cos(psi - t),  q = -rho [(2 - a + a cos t) cos psi + a sin t sin psi],
//   rho = (2 sin(t/2))^a, psi = a (t - pi)/2.
__device__ double symbol_sample(double a, int weights, int j, int Np) {
    const double u = (double)j / (double)Np;        // t / pi
    const double rho = pow(2.0 * sinpi(0.5 * u), a);
    const double psi = 0.5 * a * (u - 1.0);         // psi / pi
    if (weights == FDE_WEIGHTS_GL1) return -2.0 * rho * cospi(psi - u);
    return -rho * ((2.0 - a + a * cospi(u)) * cospi(psi) + a * sinpi(u) * sinpi(psi));
}

// Weights w_0..w_{n+1} and the first column of the L-circulant embedding of
// T, packed into bufA (one CTA: the weights' prefix product is a block scan).
__device__ void axis_weights_and_column(const AxisJob& J) {
    const int n = J.n, Np = J.Np;
    const int L = 2 * Np;
    {
        // g_k = (-1)^k binom(alpha, k) = f_1 f_2 ... f_k with
        // f_i = -(alpha - i + 1) / i, as a parallel prefix product: each thread
        // multiplies the factors of its chunk of k, a block scan gives each
        // thread the product of all earlier chunks, and the thread then forms
        // its g_k in order.  WSGD: w_k = (alpha/2) g_k + ((2-alpha)/2) g_{k-1}.
        __shared__ double scan[1024];
        const int K = n + 1;
        const int nt = blockDim.x;
        const int c = (K + nt - 1) / nt;
        const int k0 = (int)threadIdx.x * c + 1;
        const int k1 = k0 + c - 1 < K ? k0 + c - 1 : K;
        double p = 1.0;
        for (int k = k0; k <= k1; ++k) p *= -(J.alpha - k + 1.0) / k;
        scan[threadIdx.x] = p;
        __syncthreads();
        for (int off = 1; off < nt; off <<= 1) {
            const double v = (int)threadIdx.x >= off ? scan[threadIdx.x - off] : 1.0;
            __syncthreads();
            scan[threadIdx.x] *= v;
            __syncthreads();
        }
        double g = threadIdx.x > 0 ? scan[threadIdx.x - 1] : 1.0;     // g_{k0 - 1}
        const bool gl1 = J.weights == FDE_WEIGHTS_GL1;
        if (threadIdx.x == 0) J.wts[0] = gl1 ? 1.0 : 0.5 * J.alpha;
        for (int k = k0; k <= k1; ++k) {
            const double gprev = g;
            g *= -(J.alpha - k + 1.0) / k;
            J.wts[k] = gl1 ? g : 0.5 * J.alpha * g + 0.5 * (2.0 - J.alpha) * gprev;
        }
    }
    __syncthreads();
    // first column of the L-circulant embedding T: c_k = -w_{k+1} (k < n), c_{L-1} = -w_0
    for (int m = threadIdx.x; m < Np; m += blockDim.x) {
        double c[2];
        for (int e = 0; e < 2; ++e) {
            const int k = 2 * m + e;
            c[e] = k < n ? -J.wts[k + 1] : (k == L - 1 ? -J.wts[0] : 0.0);
        }
        J.bufA[m] = mk(c[0], c[1]);
    }
}

// lambda_j / L from the packed transform Z for the pair (j, Np - j), both
// precisions.
__device__ void axis_lambda_pair(const AxisJob& J, const cx<double>* Z, int j) {
    const int Np = J.Np;
    const int wsh = J.logTW - (J.logNp + 1);
    const double invL = 1.0 / (double)(2 * Np);
    const int jm = (Np - j) & (Np - 1);
    cx<double> a, b;
    unpack_pair(Z[j], Z[jm], J.tw64[j << wsh], a, b);
    const cx<double> la = invL * a, lb = invL * conj(b);
    J.lam64[j] = la;
    J.lam32[j] = mk((float)la.x, (float)la.y);
    J.lam64[Np - j] = lb;
    J.lam32[Np - j] = mk((float)lb.x, (float)lb.y);
}

// The tau multiplier (or 2D axis part) at frequency j.
__device__ void axis_phi(const AxisJob& J, int j) {
    const int n = J.n, Np = J.Np;
    const double invL = 1.0 / (double)(2 * Np);
    double v = 0.0;
    if (j >= 1 && j <= n) {
        const double F = symbol_sample(J.alpha, J.weights, j, Np);
        if (J.kind == 0 && J.dbar) {
            v = invL / (F + J.add / *J.dbar);
        } else if (J.kind == 0 && J.fold_d) {
            const double Dj = 0.5 * ((J.dp ? J.dp[j - 1] : J.dpc) + (J.dm ? J.dm[j - 1] : J.dmc));
            v = invL / (Dj * F);
        } else {
            v = J.kind == 0 ? invL / (J.add + J.mult * F) : J.add + J.mult * F;
        }
    }
    J.phi64[j] = v;
    J.phi32[j] = (float)v;
}

// A short axis in one CTA: weights, the ping-pong FFT, lambda and the
// multiplier samples.
__global__ void __launch_bounds__(1024) k_axis(AxisJob J) {
    axis_weights_and_column(J);
    __syncthreads();
    cx<double>* Z = fft_pingpong<double, false>(J.bufA, J.bufB, J.logNp, J.tw64, J.logTW);
    for (int j = threadIdx.x; j <= J.Np / 2; j += blockDim.x) axis_lambda_pair(J, Z, j);
    for (int j = threadIdx.x; j <= J.Np; j += blockDim.x) axis_phi(J, j);
}

// A long axis across the GPU: the weights in one CTA, then every radix pass of
// the ping-pong FFT, the lambda pairs and the multiplier samples (one
// transcendental-heavy FP64 evaluation per frequency) as grid-wide launches.
// One CTA took 4.4 ms for Np = 65536, most of it in the samples.
__global__ void __launch_bounds__(1024) k_axis_weights(AxisJob J) { axis_weights_and_column(J); }

template <int RAD>
__global__ void k_axis_fft_pass(const cx<double>* src, cx<double>* dst, int logP, int logNs, const cx<double>* tw,
                                int logTW) {
    constexpr int LR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
    const int logItems = logP - LR;
    const int items = 1 << logItems;
    const int twsh = logTW - logNs - LR;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < items; j += gridDim.x * blockDim.x)
        stockham_item_pp<double, RAD, false>(src, dst, j, logItems, 1 << logNs, twsh, tw);
}

__global__ void k_axis_spectrum(AxisJob J, const cx<double>* Z) {
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= J.Np / 2; j += stride) axis_lambda_pair(J, Z, j);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= J.Np; j += stride) axis_phi(J, j);
}

// Lines of at least this many packed points take the grid-wide path.
constexpr int kAxisGridNp = 8192;

void launch_axis(const AxisJob& J, int num_sms, cudaStream_t st) {
    if (J.Np < kAxisGridNp) {
        k_axis<<<1, 1024, 0, st>>>(J);
        return;
    }
    k_axis_weights<<<1, 1024, 0, st>>>(J);
    const int blocks = num_sms > 0 ? num_sms : 1;
    cx<double>* src = J.bufA;
    cx<double>* dst = J.bufB;
    int logNs = 0;
    for (int rem = J.logNp; rem > 0;) {
        const int lr = rem >= 3 ? 3 : rem;
        if (lr == 3) k_axis_fft_pass<8><<<blocks, 256, 0, st>>>(src, dst, J.logNp, logNs, J.tw64, J.logTW);
        else if (lr == 2) k_axis_fft_pass<4><<<blocks, 256, 0, st>>>(src, dst, J.logNp, logNs, J.tw64, J.logTW);
        else k_axis_fft_pass<2><<<blocks, 256, 0, st>>>(src, dst, J.logNp, logNs, J.tw64, J.logTW);
        logNs += lr;
        rem -= lr;
        cx<double>* t = src;
        src = dst;
        dst = t;
    }
    k_axis_spectrum<<<blocks, 256, 0, st>>>(J, src);
}

struct VecJob {
    long long N;
    int dim, has_D;
    const double *dp, *dm, *ep, *em;
    double dpc, dmc, epc, emc;
    double* dinv64;
    float* dinv32;
    float *dp32, *dm32, *ep32, *em32;
};

__global__ void k_vectors(VecJob J) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < J.N;
         i += (long long)gridDim.x * blockDim.x) {
        const double dp = J.dp ? J.dp[i] : J.dpc;
        const double dm = J.dm ? J.dm[i] : J.dmc;
        if (J.dp32) J.dp32[i] = (float)dp;
        if (J.dm32 && J.dm32 != J.dp32) J.dm32[i] = (float)dm;
        double D;
        if (J.dim == 2) {
            const double ep = J.ep ? J.ep[i] : J.epc;
            const double em = J.em ? J.em[i] : J.emc;
            if (J.ep32) J.ep32[i] = (float)ep;
            if (J.em32 && J.em32 != J.ep32) J.em32[i] = (float)em;
            D = 0.25 * (dp + dm + ep + em);
        } else {
            D = 0.5 * (dp + dm);
        }
        if (J.has_D) {
            const double di = 1.0 / D;
            J.dinv64[i] = di;
            J.dinv32[i] = (float)di;
        }
    }
}

// dbar = mean of D = (d_+ + d_-)/2 over the line, in a fixed summation order
// (one block: strided per-thread sums, then a shared-memory tree).
__global__ void __launch_bounds__(1024) k_mean_d(long long N, const double* dp, const double* dm, double dpc,
                                                 double dmc, double* dbar) {
    __shared__ double red[1024];
    double s = 0.0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) s += 0.5 * ((dp ? dp[i] : dpc) + (dm ? dm[i] : dmc));
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *dbar = red[0] / (double)N;
}

// P_tri (Sec. 4, Table 2): the three main diagonals of M = c0 I + D_+ T + D_- T^T,
// T_ij = -w_{i-j+1}: M[i,i] = c0 - (d+ + d-) w_1, M[i,i+1] = -d+ w_0 - d- w_2,
// M[i,i-1] = -d+ w_2 - d- w_0, from the weights k_axis wrote.  Layout
// [lower | diagonal | upper], FP64 and FP32.
struct TriJob {
    long long n;
    double c0;
    const double *dp, *dm;
    double dpc, dmc;
    const double* wts;
    double* tri64;
    float* tri32;
};

__global__ void k_tri(TriJob J) {
    const double w0 = J.wts[0], w1 = J.wts[1], w2 = J.n >= 2 ? J.wts[2] : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < J.n;
         i += (long long)gridDim.x * blockDim.x) {
        const double dp = J.dp ? J.dp[i] : J.dpc;
        const double dm = J.dm ? J.dm[i] : J.dmc;
        const double lo = i > 0 ? -dp * w2 - dm * w0 : 0.0;
        const double di = J.c0 - (dp + dm) * w1;
        const double up = i + 1 < J.n ? -dp * w0 - dm * w2 : 0.0;
        J.tri64[i] = lo;
        J.tri64[J.n + i] = di;
        J.tri64[2 * J.n + i] = up;
        J.tri32[i] = (float)lo;
        J.tri32[J.n + i] = (float)di;
        J.tri32[2 * J.n + i] = (float)up;
    }
}

__global__ void k_write_inst(Inst v, Inst* dst) { *dst = v; }

// b = a u + c f (f may be null).
__global__ void k_step_rhs(long long N, double a, double c, const double* u, const double* f, double* b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        b[i] = a * u[i] + (f ? c * f[i] : 0.0);
}

// Team sizes for one batched solve: instance i gets a share of the G CTAs in
// proportion to cost[i] times the iteration count its previous solve left in
// info[i] (at least one CTA each).  One thread; writes team_start[0..count].
struct BalanceJob {
    int count, G;
    const fde_solve_info* info;
    SyncArea* sync;
    float cost[kMaxBatch];
};

__global__ void k_balance(const __grid_constant__ BalanceJob J) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double w[kMaxBatch];
    int ts[kMaxBatch];
    double W = 0.0;
    for (int i = 0; i < J.count; ++i) {
        int it = J.info[i].iterations;
        if (it < 1 || it > 1000000) it = 1;
        w[i] = (double)J.cost[i] * (double)it;
        W += w[i];
    }
    int used = 0;
    for (int i = 0; i < J.count; ++i) {
        int v = (int)((double)J.G * w[i] / W);
        ts[i] = v < 1 ? 1 : v;
        used += ts[i];
    }
    while (used > J.G) {                  // the one-CTA floor overshot: shrink the largest
        int b = 0;
        for (int i = 1; i < J.count; ++i) if (ts[i] > ts[b]) b = i;
        if (ts[b] <= 1) break;
        --ts[b];
        --used;
    }
    while (used < J.G) {                  // spare CTAs to the most loaded team per CTA
        int b = 0;
        for (int i = 1; i < J.count; ++i) if (w[i] * ts[b] > w[b] * ts[i]) b = i;
        ++ts[b];
        ++used;
    }
    int acc = 0;
    for (int i = 0; i < J.count; ++i) {
        J.sync->team_start[i] = (unsigned short)acc;
        acc += ts[i];
    }
    J.sync->team_start[J.count] = (unsigned short)acc;
}

template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<unsigned char*>(ws) + off); }

// Largest FFT a CTA runs for this problem, capped for the shared twiddle table.
int twiddle_log(const fde_problem* p, const Layout& Lo, int line_mode64, int line_mode32) {
    int lg = 2;
    if (p->dim == 2) {
        lg = std::max(ilog2(Lo.Np[0]), ilog2(Lo.Np[1]));
    } else {
        const int logNp = ilog2(Lo.Np[0]);
        const int logP2 = logNp - logNp / 2;
        const bool any_cta = line_mode64 == kLineCta || line_mode32 == kLineCta;
        lg = any_cta ? logNp : logP2;
    }
    if (lg > kMaxLogTsm) lg = kMaxLogTsm;
    return lg < 2 ? 2 : lg;
}

int line_modes(const fde_problem* p, const Layout& Lo, int work_bytes) {
    if (p->dim == 2) return kPlane | (kPlane << 8);
    const int Np = Lo.Np[0];
    const bool sym = p->dp == p->dm && (p->dp != nullptr || p->dp_const == p->dm_const);
    const int nbuf = sym ? 1 : 2;
    // a whole line in one CTA: one FFT item per thread and the buffers in shared memory
    // P_tri's shared-memory cyclic reduction holds four real vectors of the line
    const bool tri = p->order == FDE_ORDER_TRI;
    auto fits = [&](int esz) {
        return fft_lines_per_call(ilog2(Np), kThreads, esz / 2) >= 1 &&
               (long long)padded_len(Np * nbuf) * esz <= work_bytes &&
               (!tri || ((long long)4 * Np * (esz / 2) <= work_bytes && Np <= kTriCtaItems * kThreads));
    };
    const int m64 = fits((int)sizeof(cx<double>)) ? kLineCta : kLineSplit;
    const int m32 = fits((int)sizeof(cx<float>)) ? kLineCta : kLineSplit;
    return m64 | (m32 << 8);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

void fde_default_opts(fde_solve_opts* o) {
    if (!o) return;
    o->method = FDE_GMRES;
    o->restart = 30;
    o->tol = 1e-8;
    o->max_iters = 5000;
    o->precision = FDE_PREC_F64;
    o->inner_tol = 1e-4;
    o->max_outer = 50;
    o->side = FDE_SIDE_RIGHT;
    o->balance = 0;
}

const char* fde_status_string(int s) {
    switch (s) {
        case FDE_OK: return "ok";
        case FDE_EINVAL: return "invalid argument";
        case FDE_ENOMEM: return "workspace too small";
        case FDE_ECUDA: return "CUDA error";
        case FDE_ENOCONV: return "no convergence within the iteration cap";
        case FDE_EBREAKDOWN: return "Krylov breakdown";
        case FDE_ETIMEOUT: return "inter-CTA barrier timed out";
        case FDE_ENONFINITE: return "non-finite value in a reduction";
        default: return "unknown status";
    }
}

fde_status fde_workspace_size(const fde_problem* prob, const fde_solve_opts* opts, size_t* bytes) {
    if (!bytes) return FDE_EINVAL;
    const fde_status s = validate(prob, opts);
    if (s != FDE_OK) return s;
    *bytes = layout(prob, opts).total;
    return FDE_OK;
}

fde_status fde_assemble_symbol(const fde_problem* prob, const fde_solve_opts* opts, void* workspace, size_t bytes,
                               fde_plan** plan_out, void* stream) {
    if (!plan_out || !workspace) return FDE_EINVAL;
    *plan_out = nullptr;
    fde_status s = validate(prob, opts);
    if (s != FDE_OK) return s;
    if ((reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)) != 0) return FDE_EINVAL;
    const Layout Lo = layout(prob, opts);
    if (bytes < Lo.total) return FDE_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDE_ECUDA;
    DeviceInfo* di = nullptr;
    if (prepare_device(dev, &di) != cudaSuccess) return FDE_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    fde_plan* p = new (std::nothrow) fde_plan();
    if (!p) return FDE_ENOMEM;
    p->prob = *prob;
    p->opts = *opts;
    p->ws = workspace;
    p->ws_bytes = bytes;
    p->device = dev;
    p->smem_bytes = di->smem_bytes;
    for (int i = 0; i < 3; ++i) p->grid[i] = di->grid[i];

    const int m = opts->method == FDE_GMRES ? opts->restart : 1;
    // line modes against the shared memory left beside the largest twiddle table
    const int work_bytes = di->smem_bytes - (int)kshared_bytes(m, kMaxLogTsm);

    Inst& I = p->inst;
    std::memset(&I, 0, sizeof(Inst));
    I.dim = prob->dim;
    I.n1 = prob->n1;
    I.n2 = prob->dim == 2 ? prob->n2 : 1;
    I.N = (long long)I.n1 * I.n2;
    I.line_mode = line_modes(prob, Lo, work_bytes);
    I.symx = prob->dp == prob->dm && (prob->dp != nullptr || prob->dp_const == prob->dm_const);
    I.symy = prob->dim == 2 && prob->ep == prob->em && (prob->ep != nullptr || prob->ep_const == prob->em_const);
    I.has_D = Lo.has_D;
    I.order = prob->order;
    I.shift = prob->tau_shift;
    I.weights = prob->weights;
    I.method = opts->method;
    I.precision = opts->precision;
    I.restart = opts->method == FDE_GMRES ? opts->restart : 0;
    const double h1 = prob->len1 / (prob->n1 + 1);
    const double ha = std::pow(h1, prob->alpha);
    I.h_alpha = ha;
    I.c0 = (prob->scheme == FDE_SCHEME_CRANK_NICOLSON ? 2.0 : 1.0) * ha / prob->dt;
    if (prob->dim == 2) {
        const double h2 = prob->len2 / (prob->n2 + 1);
        I.sr = ha / std::pow(h2, prob->beta);
        I.phi_scale2d = 1.0 / ((double)(prob->n1 + 1) * (double)(prob->n2 + 1));
    }
    I.logTW = Lo.logTW;
    I.logTsm = twiddle_log(prob, Lo, I.line_mode & 0xff, (I.line_mode >> 8) & 0xff);
    I.tw64 = at<cx<double>>(workspace, Lo.tw64);
    I.tw32 = at<cx<float>>(workspace, Lo.tw32);
    for (int a = 0; a < prob->dim; ++a) {
        AxisData& A = I.ax[a];
        A.n = a == 0 ? prob->n1 : prob->n2;
        A.Np = A.n + 1;
        A.logNp = ilog2(A.Np);
        A.logP1 = A.logNp / 2;
        A.logP2 = A.logNp - A.logP1;
        A.P1 = 1 << A.logP1;
        A.P2 = 1 << A.logP2;
        A.lam64 = at<cx<double>>(workspace, Lo.lam64[a]);
        A.lam32 = at<cx<float>>(workspace, Lo.lam32[a]);
        A.phi64 = at<double>(workspace, Lo.phi64[a]);
        A.phi32 = at<float>(workspace, Lo.phi32[a]);
    }
    I.dp64 = prob->dp;
    I.dm64 = prob->dm;
    I.ep64 = prob->dim == 2 ? prob->ep : nullptr;
    I.em64 = prob->dim == 2 ? prob->em : nullptr;
    I.dpc = prob->dp_const;
    I.dmc = prob->dm_const;
    I.epc = prob->ep_const;
    I.emc = prob->em_const;
    I.dp32 = Lo.dp32 ? at<float>(workspace, Lo.dp32) : nullptr;
    I.dm32 = Lo.dm32 ? at<float>(workspace, Lo.dm32) : nullptr;
    I.ep32 = Lo.ep32 ? at<float>(workspace, Lo.ep32) : nullptr;
    I.em32 = Lo.em32 ? at<float>(workspace, Lo.em32) : nullptr;
    I.dinv64 = Lo.has_D ? at<double>(workspace, Lo.dinv64) : nullptr;
    I.dinv32 = Lo.has_D ? at<float>(workspace, Lo.dinv32) : nullptr;
    const bool tri = prob->order == FDE_ORDER_TRI;
    I.tri64 = tri ? at<double>(workspace, Lo.tri64) : nullptr;
    I.tri32 = tri ? at<float>(workspace, Lo.tri32) : nullptr;
    I.trisc = tri ? at<void>(workspace, Lo.trisc) : nullptr;
    I.wvec = at<void>(workspace, Lo.wvec);
    I.r64 = at<double>(workspace, Lo.r64);
    I.t64 = at<double>(workspace, Lo.t64);
    I.split64 = at<void>(workspace, Lo.split64);
    I.split32 = at<void>(workspace, Lo.split32);
    p->inst_dev = at<Inst>(workspace, Lo.inst);
    p->sync_dev = at<SyncArea>(workspace, Lo.sync);

    // --- device assembly, all on `st` ---
    k_twiddles<<<std::min(1024, (Lo.TW + 255) / 256), 256, 0, st>>>(const_cast<cx<double>*>(I.tw64),
                                                                     const_cast<cx<float>*>(I.tw32), Lo.TW);
    const bool shift = prob->tau_shift != 0;
    const double dbar = 0.5 * (prob->dp_const + prob->dm_const);
    const double ebar = 0.5 * (prob->ep_const + prob->em_const);
    for (int a = 0; a < prob->dim; ++a) {
        AxisJob J{};
        const AxisData& A = I.ax[a];
        J.n = A.n;
        J.Np = A.Np;
        J.logNp = A.logNp;
        J.logTW = Lo.logTW;
        J.weights = prob->weights;
        J.alpha = a == 0 ? prob->alpha : prob->beta;
        if (prob->dim == 1) {
            // P_F (Sec. 3.1): 1/(L F); Case I (Sec. 3.1.1): D tau(F + 2 nu/(d_+ + d_-)) = tau(nu + dbar F);
            // with variable coefficients the shift nu/mean(D) stays beside D
            J.kind = 0;
            J.add = shift ? I.c0 : 0.0;
            J.mult = shift ? dbar : 1.0;
            if (prob->order == FDE_ORDER_TAU_DF) {
                J.fold_d = 1;
                J.dp = prob->dp;
                J.dm = prob->dm;
                J.dpc = prob->dp_const;
                J.dmc = prob->dm_const;
            }
            if (shift && (prob->dp || prob->dm)) {
                double* dbar_dev = at<double>(workspace, Lo.dbar);
                k_mean_d<<<1, 1024, 0, st>>>(I.N, prob->dp, prob->dm, prob->dp_const, prob->dm_const, dbar_dev);
                J.dbar = dbar_dev;
                J.mult = 1.0;
            }
        } else {
            // Sec. 3.2: F = F_a + sr F_b, or P_hat's c0 + d F_a + sr e F_b, split per axis
            J.kind = 1;
            if (a == 0) { J.add = shift ? I.c0 : 0.0; J.mult = shift ? dbar : 1.0; }
            else { J.add = 0.0; J.mult = shift ? I.sr * ebar : I.sr; }
        }
        J.tw64 = I.tw64;
        J.lam64 = const_cast<cx<double>*>(A.lam64);
        J.lam32 = const_cast<cx<float>*>(A.lam32);
        J.phi64 = const_cast<double*>(A.phi64);
        J.phi32 = const_cast<float*>(A.phi32);
        J.wts = at<double>(workspace, Lo.wts);
        J.bufA = at<cx<double>>(workspace, Lo.split64);
        J.bufB = J.bufA + std::max(Lo.Np[0], Lo.Np[1]);
        launch_axis(J, di->num_sms, st);
    }
    VecJob V{};
    V.N = I.N;
    V.dim = prob->dim;
    V.has_D = Lo.has_D;
    V.dp = prob->dp;
    V.dm = prob->dm;
    V.ep = I.ep64;
    V.em = I.em64;
    V.dpc = prob->dp_const;
    V.dmc = prob->dm_const;
    V.epc = prob->ep_const;
    V.emc = prob->em_const;
    V.dinv64 = const_cast<double*>(I.dinv64);
    V.dinv32 = const_cast<float*>(I.dinv32);
    V.dp32 = const_cast<float*>(I.dp32);
    V.dm32 = const_cast<float*>(I.dm32);
    V.ep32 = const_cast<float*>(I.ep32);
    V.em32 = const_cast<float*>(I.em32);
    const int vblocks = (int)std::min<long long>(4096, (I.N + 255) / 256);
    k_vectors<<<vblocks, 256, 0, st>>>(V);
    if (tri) {
        TriJob T{};
        T.n = I.N;
        T.c0 = I.c0;
        T.dp = prob->dp;
        T.dm = prob->dm;
        T.dpc = prob->dp_const;
        T.dmc = prob->dm_const;
        T.wts = at<double>(workspace, Lo.wts);
        T.tri64 = const_cast<double*>(I.tri64);
        T.tri32 = const_cast<float*>(I.tri32);
        k_tri<<<vblocks, 256, 0, st>>>(T);
    }
    k_write_inst<<<1, 1, 0, st>>>(I, p->inst_dev);
    if (cudaGetLastError() != cudaSuccess) {
        delete p;
        return FDE_ECUDA;
    }
    *plan_out = p;
    return FDE_OK;
}

void fde_plan_destroy(fde_plan* p) { delete p; }

fde_status fde_plan_scalars(const fde_plan* p, double* c0, double* sr, double* h_alpha) {
    if (!p) return FDE_EINVAL;
    if (c0) *c0 = p->inst.c0;
    if (sr) *sr = p->inst.sr;
    if (h_alpha) *h_alpha = p->inst.h_alpha;
    return FDE_OK;
}

static fde_status launch_op(const fde_plan* p, int op, int dtype, const void* in, void* out, void* stream) {
    if (!p || !in || !out || in == out) return FDE_EINVAL;
    if (dtype != FDE_F64 && dtype != FDE_F32) return FDE_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EngineArgs* a = new (std::nothrow) EngineArgs();
    if (!a) return FDE_ENOMEM;
    a->op = op;
    a->count = 1;
    a->dtype = dtype;
    a->smem_bytes = p->smem_bytes;
    a->sync = p->sync_dev;
    a->info = nullptr;
    a->inst[0] = p->inst_dev;
    a->in[0] = in;
    a->out[0] = out;
    a->order[0] = 0;
    const int mode = dtype == FDE_F64 ? kModeF64 : kModeF32;
    const int lm = dtype == FDE_F64 ? (p->inst.line_mode & 0xff) : ((p->inst.line_mode >> 8) & 0xff);
    int grid = p->grid[mode];
    if (p->ctas > 0 && p->ctas < grid) grid = p->ctas;
    if (p->inst.dim == 1 && lm == kLineCta) grid = 1;
    a->team_size = grid;
    cudaError_t e = cudaMemsetAsync(p->sync_dev, 0, offsetof(SyncArea, partial), st);
    if (e == cudaSuccess) e = mode == kModeF64 ? engine_launch_f64(*a, grid, st) : engine_launch_f32(*a, grid, st);
    delete a;
    return e == cudaSuccess ? FDE_OK : FDE_ECUDA;
}

fde_status fde_toeplitz_matvec(const fde_plan* p, int dtype, const void* x, void* y, void* stream) {
    return launch_op(p, kOpMatvec, dtype, x, y, stream);
}

fde_status fde_tau_solve(const fde_plan* p, int dtype, const void* r, void* z, void* stream) {
    return launch_op(p, kOpTau, dtype, r, z, stream);
}

fde_status fde_krylov_solve(const fde_plan* const* plans, int count, const double* const* b, double* const* x,
                            const fde_solve_opts* opts, fde_solve_info* info_dev, void* stream) {
    if (!plans || !b || !x || !opts || !info_dev || count < 1 || count > kMaxBatch) return FDE_EINVAL;
    const fde_plan* p0 = plans[0];
    if (!p0) return FDE_EINVAL;
    for (int i = 0; i < count; ++i) {
        const fde_plan* p = plans[i];
        if (!p || !b[i] || !x[i] || (const void*)b[i] == (const void*)x[i]) return FDE_EINVAL;
        if (p->opts.method != p0->opts.method || p->opts.precision != p0->opts.precision ||
            p->opts.restart != p0->opts.restart || p->device != p0->device)
            return FDE_EINVAL;
    }
    if (!(opts->tol > 0.0) || opts->max_iters < 1 || (opts->side != FDE_SIDE_RIGHT && opts->side != FDE_SIDE_LEFT))
        return FDE_EINVAL;
    if (p0->opts.precision == FDE_PREC_F32_IR && (!(opts->inner_tol > 0.0) || opts->max_outer < 1)) return FDE_EINVAL;
    if (opts->balance != 0 && opts->balance != 1) return FDE_EINVAL;
    const int mode = p0->opts.precision;
    EngineArgs* a = new (std::nothrow) EngineArgs();
    if (!a) return FDE_ENOMEM;
    a->op = kOpSolve;
    a->count = count;
    a->dtype = FDE_F64;
    a->smem_bytes = p0->smem_bytes;
    a->sync = p0->sync_dev;
    a->info = info_dev;
    a->tol = opts->tol;
    a->inner_tol = opts->inner_tol;
    a->max_iters = opts->max_iters;
    a->max_outer = opts->max_outer;
    a->side = opts->side;
    bool all_cta = true;
    std::vector<int> idx(count);
    for (int i = 0; i < count; ++i) {
        const fde_plan* p = plans[i];
        a->inst[i] = p->inst_dev;
        a->in[i] = b[i];
        a->out[i] = x[i];
        idx[i] = i;
        const int lm = mode == FDE_PREC_F64 ? (p->inst.line_mode & 0xff) : ((p->inst.line_mode >> 8) & 0xff);
        if (!(p->inst.dim == 1 && lm == kLineCta)) all_cta = false;
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int u, int v) { return plans[u]->inst.N > plans[v]->inst.N; });
    for (int i = 0; i < count; ++i) a->order[i] = (unsigned short)idx[i];
    const int G = p0->grid[mode];
    int grid, ts;
    if (all_cta) {
        ts = 1;
        grid = std::min(G, count);
    } else if (count >= G) {
        ts = 1;
        grid = G;
    } else if (count == 1 && p0->ctas > 0 && p0->ctas < G) {
        ts = p0->ctas;          // a schedule chosen by fde_plan_set_schedule / fde_autotune
        grid = ts;
    } else {
        ts = G / count;
        grid = ts * count;
    }
    a->team_size = ts;
    a->team_mode = 0;
    const bool balanced = opts->balance == 1 && !all_cta && count > 1 && count < G;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(p0->sync_dev, 0, offsetof(SyncArea, partial), st);
    if (e == cudaSuccess && balanced) {
        BalanceJob* B = new (std::nothrow) BalanceJob();
        if (!B) {
            delete a;
            return FDE_ENOMEM;
        }
        B->count = count;
        B->G = G;
        B->info = info_dev;
        B->sync = p0->sync_dev;
        for (int i = 0; i < count; ++i) {
            const Inst& I = plans[i]->inst;
            double c = 0.0;
            for (int ax = 0; ax < I.dim; ++ax) c += (double)I.N * (I.ax[ax].logNp + 1);
            B->cost[i] = (float)c;
        }
        k_balance<<<1, 32, 0, st>>>(*B);
        delete B;
        e = cudaGetLastError();
        a->team_mode = 1;
        grid = G;
    }
    if (e == cudaSuccess) {
        if (mode == FDE_PREC_F64) e = engine_launch_f64(*a, grid, st);
        else if (mode == FDE_PREC_F32) e = engine_launch_f32(*a, grid, st);
        else e = engine_launch_ir(*a, grid, st);
    }
    delete a;
    return e == cudaSuccess ? FDE_OK : FDE_ECUDA;
}

fde_status fde_step_rhs(const fde_plan* p, const double* u_prev, const double* f, double* b, void* stream) {
    if (!p || !u_prev || !b || u_prev == b) return FDE_EINVAL;
    const long long N = p->inst.N;
    const int blocks = (int)std::min<long long>(4096, (N + 255) / 256);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->prob.scheme == FDE_SCHEME_IMPLICIT_EULER) {
        k_step_rhs<<<blocks, 256, 0, st>>>(N, p->inst.c0, p->inst.h_alpha, u_prev, f, b);
        return cudaGetLastError() == cudaSuccess ? FDE_OK : FDE_ECUDA;
    }
    // Crank-Nicolson: the explicit half, b = (2 c0 I - M) u_prev + 2 h^alpha f
    k_step_rhs<<<blocks, 256, 0, st>>>(N, 2.0 * p->inst.c0, 2.0 * p->inst.h_alpha, u_prev, f, b);
    if (cudaGetLastError() != cudaSuccess) return FDE_ECUDA;
    return launch_op(p, kOpMatvecSub, FDE_F64, u_prev, b, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// fde_toeplitz_matvec_noalloc: y = M x for a 1D problem with its symbol data
// and transform buffers in a fixed static device array instead of a
// caller-provided workspace.
// ---------------------------------------------------------------------------

namespace {

constexpr int kNoallocMaxNp = FDE_MATVEC_NOALLOC_MAX_N + 1;   // 4096: L = 8192
constexpr int kNoallocTW = 2 * kNoallocMaxNp;

struct NoallocLayout {
    size_t tw64, tw32, lam64, lam32, phi64, phi32, wts, buf, total;
};

constexpr NoallocLayout noalloc_layout() {
    NoallocLayout L{};
    size_t off = 0;
    auto take = [&off](size_t b) { const size_t o = off; off = (off + b + kAlign - 1) & ~(kAlign - 1); return o; };
    L.tw64 = take((size_t)kNoallocTW * sizeof(cx<double>));
    L.tw32 = take((size_t)kNoallocTW * sizeof(cx<float>));
    L.lam64 = take((size_t)(kNoallocMaxNp + 1) * sizeof(cx<double>));
    L.lam32 = take((size_t)(kNoallocMaxNp + 1) * sizeof(cx<float>));
    L.phi64 = take((size_t)(kNoallocMaxNp + 1) * sizeof(double));
    L.phi32 = take((size_t)(kNoallocMaxNp + 1) * sizeof(float));
    L.wts = take((size_t)(kNoallocMaxNp + 2) * sizeof(double));
    L.buf = take((size_t)4 * kNoallocMaxNp * sizeof(cx<double>));   // two ping-pong pairs
    L.total = off;
    return L;
}

constexpr NoallocLayout kNoalloc = noalloc_layout();
static_assert(kNoalloc.total == FDE_MATVEC_NOALLOC_SCRATCH_BYTES, "scratch size in fde.h is stale");

}  // namespace

// The scratch itself: file scope, one copy per device.
static __device__ __align__(256) unsigned char g_matvec_scratch[FDE_MATVEC_NOALLOC_SCRATCH_BYTES];

namespace {

// The driver's context calls, reached through the runtime (no link against
// the driver library).  cuCtxGetId gives an id that is unique for the
// process's lifetime, so a context created after cudaDeviceReset never
// matches one whose module instance has gone, even if its handle is reused.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct ScratchSlot {
    unsigned long long ctx_id;   // 0: not resolved
    unsigned char* ptr;
};

std::mutex g_scratch_mu;
ScratchSlot g_scratch[64];
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the context current on this thread, 0 if none is current yet.
cudaError_t current_context_id(unsigned long long* id) {
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
    if (!ctx) return cudaSuccess;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

// Device address of g_matvec_scratch in the context current on `dev`: resolved
// with cudaGetSymbolAddress on the first call in that context (once per device
// in normal use) and cached under the context's id.
cudaError_t matvec_scratch(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    ScratchSlot& slot = g_scratch[dev];
    if (id == 0 || slot.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_matvec_scratch);   // makes the primary context current if none was
        if (e != cudaSuccess) return e;
        if (id == 0) {
            e = current_context_id(&id);
            if (e != cudaSuccess) return e;
        }
        slot.ctx_id = id;
        slot.ptr = static_cast<unsigned char*>(p);
    }
    *out = slot.ptr;
    return cudaSuccess;
}

struct LineJob {
    int n, Np, logNp, logTW;
    double c0;
    const double* dp;
    const double* dm;
    double dpc, dmc;
    const cx<double>* tw64;
    const cx<double>* lam;     // circulant eigenvalues / L, [Np + 1]
    const double* x;
    double* y;
    cx<double>* buf;           // 4 Np complex values
};

// One CTA: the zero-extended line x (v_k = x_k for 1 <= k <= n, 0 elsewhere on
// 0..L-1) is packed, transformed, multiplied by lambda and by conj(lambda)
// (T x and T^T x) and transformed back; y = c0 x + d_+ T x + d_- T^T x.
__global__ void __launch_bounds__(1024) k_line_matvec(LineJob J) {
    const int n = J.n, Np = J.Np;
    cx<double>* A = J.buf;
    cx<double>* B = A + Np;
    cx<double>* C = B + Np;
    cx<double>* D = C + Np;
    for (int m = threadIdx.x; m < Np; m += blockDim.x) {
        const int k0 = 2 * m, k1 = 2 * m + 1;
        A[m] = mk(k0 >= 1 && k0 <= n ? J.x[k0 - 1] : 0.0, k1 <= n ? J.x[k1 - 1] : 0.0);
    }
    __syncthreads();
    cx<double>* Z = fft_pingpong<double, false>(A, B, J.logNp, J.tw64, J.logTW);
    cx<double>* Zo = Z == A ? B : A;
    const int wsh = J.logTW - (J.logNp + 1);
    for (int j = threadIdx.x; j <= Np / 2; j += blockDim.x) {
        const int jm = (Np - j) & (Np - 1);
        const cx<double> wj = J.tw64[j << wsh];
        cx<double> a, b, Qj, Qm;
        unpack_pair(Z[j], Z[jm], wj, a, b);
        const cx<double> lj = J.lam[j];
        const cx<double> lm = J.lam[Np - j];
        repack_pair(lj * a, conj(lm) * b, wj, Qj, Qm);
        C[j] = Qj;
        if (jm != j) C[jm] = Qm;
        repack_pair(conj(lj) * a, lm * b, wj, Qj, Qm);
        Zo[j] = Qj;
        if (jm != j) Zo[jm] = Qm;
    }
    __syncthreads();
    const cx<double>* R1 = fft_pingpong<double, true>(C, D, J.logNp, J.tw64, J.logTW);
    const cx<double>* R2 = fft_pingpong<double, true>(Zo, Z, J.logNp, J.tw64, J.logTW);
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int k = p + 1;
        const cx<double> q1 = R1[k >> 1];
        const cx<double> q2 = R2[k >> 1];
        const double ta = (k & 1) ? q1.y : q1.x;
        const double tb = (k & 1) ? q2.y : q2.x;
        const double dp = J.dp ? J.dp[p] : J.dpc;
        const double dm = J.dm ? J.dm[p] : J.dmc;
        J.y[p] = J.c0 * J.x[p] + dp * ta + dm * tb;
    }
}

}  // namespace

extern "C" fde_status fde_toeplitz_matvec_noalloc(const fde_problem* prob, const double* x, double* y,
                                                  void* stream) {
    if (!prob || !x || !y || x == y) return FDE_EINVAL;
    const fde_problem* p = prob;
    if (p->dim != 1 || p->n1 < 1 || !is_pow2((long long)p->n1 + 1) || !valid_order(p->alpha)) return FDE_EINVAL;
    if (!(p->len1 > 0.0) || !std::isfinite(p->len1) || !(p->dt > 0.0) || !std::isfinite(p->dt)) return FDE_EINVAL;
    if (p->scheme != FDE_SCHEME_IMPLICIT_EULER && p->scheme != FDE_SCHEME_CRANK_NICOLSON) return FDE_EINVAL;
    if (p->weights != FDE_WEIGHTS_GL1 && p->weights != FDE_WEIGHTS_WSGD2) return FDE_EINVAL;
    if (!coeff_ok(p->dp, p->dp_const) || !coeff_ok(p->dm, p->dm_const)) return FDE_EINVAL;
    if (p->n1 > FDE_MATVEC_NOALLOC_MAX_N) return FDE_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDE_ECUDA;
    unsigned char* s = nullptr;
    if (matvec_scratch(dev, &s) != cudaSuccess) return FDE_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const int Np = p->n1 + 1;
    const int logNp = ilog2(Np);
    const int TW = std::max(2 * Np, 16);
    const int logTW = ilog2(TW);
    auto tw64 = reinterpret_cast<cx<double>*>(s + kNoalloc.tw64);
    auto lam64 = reinterpret_cast<cx<double>*>(s + kNoalloc.lam64);
    k_twiddles<<<std::min(1024, (TW + 255) / 256), 256, 0, st>>>(tw64, reinterpret_cast<cx<float>*>(s + kNoalloc.tw32),
                                                                 TW);
    AxisJob J{};
    J.n = p->n1;
    J.Np = Np;
    J.logNp = logNp;
    J.logTW = logTW;
    J.weights = p->weights;
    J.alpha = p->alpha;
    J.kind = 0;
    J.add = 0.0;
    J.mult = 1.0;
    J.tw64 = tw64;
    J.lam64 = lam64;
    J.lam32 = reinterpret_cast<cx<float>*>(s + kNoalloc.lam32);
    J.phi64 = reinterpret_cast<double*>(s + kNoalloc.phi64);
    J.phi32 = reinterpret_cast<float*>(s + kNoalloc.phi32);
    J.wts = reinterpret_cast<double*>(s + kNoalloc.wts);
    J.bufA = reinterpret_cast<cx<double>*>(s + kNoalloc.buf);
    J.bufB = J.bufA + Np;
    k_axis<<<1, 1024, 0, st>>>(J);

    LineJob M{};
    M.n = p->n1;
    M.Np = Np;
    M.logNp = logNp;
    M.logTW = logTW;
    const double ha = std::pow(p->len1 / (p->n1 + 1), p->alpha);
    M.c0 = (p->scheme == FDE_SCHEME_CRANK_NICOLSON ? 2.0 : 1.0) * ha / p->dt;
    M.dp = p->dp;
    M.dm = p->dm;
    M.dpc = p->dp_const;
    M.dmc = p->dm_const;
    M.tw64 = tw64;
    M.lam = lam64;
    M.x = x;
    M.y = y;
    M.buf = reinterpret_cast<cx<double>*>(s + kNoalloc.buf);
    k_line_matvec<<<1, 1024, 0, st>>>(M);
    return cudaGetLastError() == cudaSuccess ? FDE_OK : FDE_ECUDA;
}

// ---------------------------------------------------------------------------
// Transform schedules: CTAs per plan, and the layout of a 1D line
// ---------------------------------------------------------------------------

namespace {

// Work bytes of one CTA beside the Krylov scalars and a twiddle table of 2^logT.
int work_bytes_for(const fde_plan* p, int logT) {
    const int m = p->opts.method == FDE_GMRES ? p->opts.restart : 1;
    return p->smem_bytes - (int)kshared_bytes(m, logT);
}

// Can a line of Np = 2^(logP1 + logP2) be split as P1 x P2 in the four-step
// layout with elements of esz bytes (complex)?  Rows hold two lines plus a
// second output set; columns need at least one line.
bool split_feasible(const fde_plan* p, int logP1, int logP2, int esz) {
    if (logP1 < 4 || logP1 > logP2 || logP2 > kMaxLogTsm) return false;
    const int logT = logP2;
    const int work = work_bytes_for(p, logT);
    if (fft_lines_per_call(logP2, kThreads, esz / 2) < 1 || fft_lines_per_call(logP1, kThreads, esz / 2) < 1)
        return false;
    return (long long)padded_len(4 << logP2) * esz <= work && (long long)padded_len(2 << logP1) * esz <= work;
}

}  // namespace

extern "C" fde_status fde_plan_set_schedule(fde_plan* p, int ctas, int log_p1, void* stream) {
    if (!p || ctas < 0 || log_p1 < 0) return FDE_EINVAL;
    Inst I = p->inst;
    if (I.dim == 2) {
        if (log_p1 != 0) return FDE_EINVAL;
    } else {
        AxisData& A = I.ax[0];
        const int m = p->opts.method == FDE_GMRES ? p->opts.restart : 1;
        const int work_max = p->smem_bytes - (int)kshared_bytes(m, kMaxLogTsm);
        int lm64, lm32, logP1;
        if (log_p1 == 0) {
            // whole lines in one CTA where they fit, else the balanced split
            Layout Lo{};
            Lo.Np[0] = A.Np;
            const int lmodes = line_modes(&p->prob, Lo, work_max);
            lm64 = lmodes & 0xff;
            lm32 = (lmodes >> 8) & 0xff;
            logP1 = A.logNp / 2;
        } else {
            // both element sizes: the operator calls take either dtype on any plan
            const int logP2 = A.logNp - log_p1;
            if (!split_feasible(p, log_p1, logP2, (int)sizeof(cx<double>)) ||
                !split_feasible(p, log_p1, logP2, (int)sizeof(cx<float>)))
                return FDE_EINVAL;
            lm64 = lm32 = kLineSplit;
            logP1 = log_p1;
        }
        A.logP1 = logP1;
        A.logP2 = A.logNp - logP1;
        A.P1 = 1 << A.logP1;
        A.P2 = 1 << A.logP2;
        I.line_mode = lm64 | (lm32 << 8);
        const bool any_cta = lm64 == kLineCta || lm32 == kLineCta;
        int lg = any_cta ? A.logNp : A.logP2;
        if (lg > kMaxLogTsm) lg = kMaxLogTsm;
        I.logTsm = lg < 2 ? 2 : lg;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_write_inst<<<1, 1, 0, st>>>(I, p->inst_dev);
    if (cudaGetLastError() != cudaSuccess) return FDE_ECUDA;
    p->inst = I;
    p->ctas = ctas;
    return FDE_OK;
}

namespace {

struct TuneKey {
    int dim, n1, n2, precision, method, restart;
    bool operator<(const TuneKey& o) const {
        const int a[6] = {dim, n1, n2, precision, method, restart};
        const int b[6] = {o.dim, o.n1, o.n2, o.precision, o.method, o.restart};
        for (int i = 0; i < 6; ++i)
            if (a[i] != b[i]) return a[i] < b[i];
        return false;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;

// Mean time of one tau solve + one matvec (the operators of an iteration) in ms.
fde_status time_schedule(fde_plan* p, int dtype, void* in, void* out, cudaStream_t st, float* ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FDE_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FDE_ECUDA;
    }
    fde_status s = FDE_OK;
    const int reps = 3;
    for (int r = 0; r < 1 + reps && s == FDE_OK; ++r) {
        if (r == 1 && cudaEventRecord(e0, st) != cudaSuccess) s = FDE_ECUDA;
        if (s == FDE_OK) s = launch_op(p, kOpTau, dtype, in, out, st);
        if (s == FDE_OK) s = launch_op(p, kOpMatvec, dtype, out, in, st);
    }
    if (s == FDE_OK && cudaEventRecord(e1, st) != cudaSuccess) s = FDE_ECUDA;
    if (s == FDE_OK && cudaEventSynchronize(e1) != cudaSuccess) s = FDE_ECUDA;
    if (s == FDE_OK && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) s = FDE_ECUDA;
    if (s == FDE_OK) *ms /= (float)reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

}  // namespace

extern "C" fde_status fde_autotune(fde_plan* p, void* stream, int* ctas_out, int* log_p1_out) {
    if (!p) return FDE_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const TuneKey key{p->prob.dim, p->prob.n1, p->prob.dim == 2 ? p->prob.n2 : 1, p->opts.precision,
                      p->opts.method, p->opts.restart};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            const fde_status s = fde_plan_set_schedule(p, it->second.first, it->second.second, stream);
            if (s == FDE_OK) {
                if (ctas_out) *ctas_out = it->second.first;
                if (log_p1_out) *log_p1_out = it->second.second;
            }
            return s;
        }
    }
    const int dtype = p->opts.precision == FDE_PREC_F64 ? FDE_F64 : FDE_F32;
    const int mode = dtype == FDE_F64 ? kModeF64 : kModeF32;
    const int G = p->grid[mode];
    // scratch: the plan's FP64 residual vector (N doubles also hold N floats) and
    // its first Krylov vector; the operators' own 2D scratch is t64
    void* in = p->inst.r64;
    void* out = p->inst.wvec;
    if (cudaMemsetAsync(in, 0, (size_t)p->inst.N * sizeof(double), st) != cudaSuccess) return FDE_ECUDA;
    std::vector<int> team;
    for (int c = 16; c < G; c *= 2) team.push_back(c);
    team.push_back(G);
    std::vector<std::pair<int, int>> cand;
    if (p->inst.dim == 2) {
        for (int c : team) cand.push_back({c, 0});
    } else {
        cand.push_back({0, 0});                       // whole lines per CTA where they fit
        const int logNp = p->inst.ax[0].logNp;
        for (int l1 = 4; 2 * l1 <= logNp; ++l1)
            for (int c : team) cand.push_back({c, l1});
    }
    const int saved_ctas = p->ctas;
    const int saved_lp1 = p->inst.ax[0].logP1;
    const bool saved_split = p->inst.dim == 1 &&
        ((dtype == FDE_F64 ? p->inst.line_mode & 0xff : (p->inst.line_mode >> 8) & 0xff) == kLineSplit);
    float best = 0.0f;
    std::pair<int, int> pick{-1, -1};
    for (const auto& c : cand) {
        if (fde_plan_set_schedule(p, c.first, c.second, stream) != FDE_OK) continue;   // infeasible
        float ms = 0.0f;
        const fde_status s = time_schedule(p, dtype, in, out, st, &ms);
        if (s != FDE_OK) return s;
        if (pick.first < 0 || ms < best) {
            best = ms;
            pick = c;
        }
    }
    if (pick.first < 0) {
        fde_plan_set_schedule(p, saved_ctas, saved_split ? saved_lp1 : 0, stream);
        return FDE_ECUDA;
    }
    const fde_status s = fde_plan_set_schedule(p, pick.first, pick.second, stream);
    if (s != FDE_OK) return s;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = pick;
    }
    if (ctas_out) *ctas_out = pick.first;
    if (log_p1_out) *log_p1_out = pick.second;
    return FDE_OK;
}

// ---------------------------------------------------------------------------
// Failure-path self-test: a team barrier whose partner never arrives
// ---------------------------------------------------------------------------

namespace {

// Two CTAs, each the only member that arrives at its own team barrier (team i
// of two CTAs on the plan's sync area; the partners are never launched).  CTA
// 0 waits with a short bound, which runs out and raises the launch's abort
// flag.  CTA 1 waits with the full bound (about 2 s), but must notice the
// abort flag on its next poll and return as well.  status[i] receives CTA i's
// result.
__global__ void k_barrier_selftest(SyncArea* sync, long long short_bound, int* status) {
    const int i = blockIdx.x;
    Team t;
    t.rank = 0;
    t.size = 2;
    t.count = &sync->bar_count[i];
    t.gen = &sync->bar_gen[i];
    t.partial = sync->partial;
    t.abort_flag = &sync->abort_flag;
    t.sync = sync;
    const bool ok = team_sync(t, i == 0 ? short_bound : kBarrierCycles);
    if (threadIdx.x == 0) status[i] = ok ? FDE_OK : FDE_ETIMEOUT;
}

}  // namespace

extern "C" fde_status fde_selftest_barrier_timeout(const fde_plan* p, int* status_dev, void* stream) {
    if (!p || !status_dev) return FDE_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(p->sync_dev, 0, offsetof(SyncArea, partial), st) != cudaSuccess) return FDE_ECUDA;
    k_barrier_selftest<<<2, kThreads, 0, st>>>(p->sync_dev, 2000000LL, status_dev);
    if (cudaGetLastError() != cudaSuccess) return FDE_ECUDA;
    // leave the sync area clean for the plan's next launch
    if (cudaMemsetAsync(p->sync_dev, 0, offsetof(SyncArea, partial), st) != cudaSuccess) return FDE_ECUDA;
    return FDE_OK;
}

// ---------------------------------------------------------------------------
// FP64 FMA rate probe: the denominator of the FP64 rooflines, measured
// ---------------------------------------------------------------------------

namespace {

__device__ double g_dfma_sink;

// Eight independent FMA chains per thread; the sum is stored only if it
// equals a value it never reaches, which keeps the chains live.
__global__ void __launch_bounds__(256) k_dfma_rate(int iters, double seed) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + 1e-7 * (double)threadIdx.x + (double)k;
    const double m = 1.0000000001, c = 1e-12;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == -1.0) g_dfma_sink = s;
}

}  // namespace

extern "C" fde_status fde_measure_fp64_rate(double* tflops, void* stream) {
    if (!tflops) return FDE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDE_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FDE_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = sms * 8, threads = 256, iters = 20000;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FDE_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FDE_ECUDA;
    }
    fde_status s = FDE_OK;
    k_dfma_rate<<<blocks, threads, 0, st>>>(iters / 10, 1.0);       // warm-up
    if (cudaEventRecord(e0, st) != cudaSuccess) s = FDE_ECUDA;
    k_dfma_rate<<<blocks, threads, 0, st>>>(iters, 1.0);
    if (s == FDE_OK && cudaGetLastError() != cudaSuccess) s = FDE_ECUDA;
    if (s == FDE_OK && cudaEventRecord(e1, st) != cudaSuccess) s = FDE_ECUDA;
    float ms = 0.0f;
    if (s == FDE_OK && cudaEventSynchronize(e1) != cudaSuccess) s = FDE_ECUDA;
    if (s == FDE_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s = FDE_ECUDA;
    if (s == FDE_OK) *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}
