// Device-side types shared by the libfde kernels: complex arithmetic, the
// per-plan instance record that lives in the caller's workspace, and small
// index helpers.  Host and device see the same POD layouts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fde.h"

#define FDE_HD __host__ __device__ __forceinline__
#define FDE_D __device__ __forceinline__
#define FDE_NI __device__ __noinline__

namespace fde {

constexpr int kThreads = 512;          // threads per CTA of the persistent engine
constexpr int kMaxRestart = 64;        // GMRES(m) upper bound on m
constexpr int kMaxDots = kMaxRestart + 2;
constexpr int kMaxBatch = 1024;        // instances per fde_krylov_solve launch
constexpr int kMaxCtas = 1024;         // grid-size bound for the sync region
constexpr int kTraceEntries = 8192;    // phase timestamps of FDE_TRACE builds
constexpr int kMaxLogTsm = 12;         // shared twiddle table: up to W_4096 (16 KB quarter wave)

template <typename R>
struct alignas(2 * sizeof(R)) cx {
    R x, y;
};

template <typename R> FDE_HD cx<R> mk(R a, R b) { cx<R> z; z.x = a; z.y = b; return z; }
template <typename R> FDE_HD cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename R> FDE_HD cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename R> FDE_HD cx<R> operator*(cx<R> a, cx<R> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> FDE_HD cx<R> operator*(R s, cx<R> a) { return mk(s * a.x, s * a.y); }
template <typename R> FDE_HD cx<R> conj(cx<R> a) { return mk(a.x, -a.y); }
template <typename R> FDE_HD cx<R> mul_i(cx<R> a) { return mk(-a.y, a.x); }       // i a
template <typename R> FDE_HD cx<R> mul_mi(cx<R> a) { return mk(a.y, -a.x); }      // -i a
template <typename R> FDE_HD cx<R> czero() { return mk(R(0), R(0)); }
template <typename R> FDE_HD cx<R> cvt(cx<double> a) { return mk(R(a.x), R(a.y)); }

// Threads of a CTA that work and synchronise together: the whole CTA
// (barrier 0, the one __syncthreads uses), or one of its two halves (warps
// 0-7 or 8-15 of 512 threads, named barriers 1 and 2), whose phases then
// interleave on the SM: one half's global loads overlap the other's FFT.
struct Grp {
    int tid;    // thread index within the group
    int nt;     // threads in the group (a multiple of 32)
    int bar;    // hardware barrier id
};
FDE_D Grp grp_cta() { return Grp{(int)threadIdx.x, (int)blockDim.x, 0}; }
FDE_D Grp grp_half(int h) {
    const int nt = (int)blockDim.x / 2;
    return Grp{(int)threadIdx.x - h * nt, nt, 1 + h};
}
// Every thread of the group executes the same sequence of grp_sync calls
// (all loops over units and lines have group-uniform bounds).
FDE_D void grp_sync(const Grp& g) {
    if (g.bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(g.bar), "r"(g.nt) : "memory");
}

FDE_HD int ilog2(long long v) { int l = 0; while ((1LL << l) < v) ++l; return l; }

// Symbol data of one axis.  Np = n + 1 (a power of two) is the length of the
// packed complex FFT; the circulant that embeds the Toeplitz factor has size
// L = 2 Np.  Multipliers are stored for frequencies k = 0..Np of the L-point
// spectrum; the rest follow from Hermitian symmetry.
struct AxisData {
    int n, Np, logNp;
    int P1, P2, logP1, logP2;          // Np = P1 * P2 for lines split across CTAs
    const cx<double>* lam64;           // [Np+1] eigenvalues of the circulant / L
    const cx<float>* lam32;
    const double* phi64;               // 1D: [Np+1] tau multiplier; 2D: [Np+1] per-axis symbol part
    const float* phi32;
};

enum LineMode : int { kLineCta = 0, kLineSplit = 1, kPlane = 2 };

// Everything a kernel needs about one assembled plan.  Written once into the
// plan's workspace by the assembly kernel.
struct Inst {
    int dim, n1, n2;
    long long N;
    int line_mode;                     // LineMode
    int symx, symy;                    // d_+ == d_- (and e_+ == e_-): one real multiplier
    int has_D, order, shift, weights;
    int method, precision, restart;
    double c0, sr, h_alpha;
    double phi_scale2d;                // 2/(n1+1) / L2 folded into the 2D tau multiplier
    AxisData ax[2];
    int logTW;
    int logTsm;                        // shared-memory twiddle table covers FFTs up to 2^logTsm
    const cx<double>* tw64;            // [TW] exp(-2 pi i t / TW)
    const cx<float>* tw32;
    // diffusion coefficients: arrays (FP64 user memory, FP32 copies) or constants
    const double *dp64, *dm64, *ep64, *em64;
    const float *dp32, *dm32, *ep32, *em32;
    double dpc, dmc, epc, emc;
    const double* dinv64;              // D^{-1} or null
    const float* dinv32;
    const double* tri64;               // P_tri: [3N] lower, diagonal, upper of M (else null)
    const float* tri32;
    void* trisc;                       // P_tri on split lines: 8N elements of cyclic-reduction state
    // solver workspace
    void* wvec;                        // vectors of the working precision
    double* r64;                       // FP64 outer residual (refinement modes)
    double* t64;                       // FP64 matvec output (refinement modes)
    void* split64;                     // 2 * Np complex FP64 intermediates (split lines)
    void* split32;                     // 2 * Np complex FP32 intermediates
};

// Launch-wide synchronisation and reduction area (in plan[0]'s workspace).
struct SyncArea {
    unsigned int bar_count[kMaxCtas];  // one counter/generation pair per team
    unsigned int bar_gen[kMaxCtas];
    unsigned int queue;                // dynamic instance queue for one-CTA teams
    unsigned int abort_flag;
    unsigned int trace_n;              // FDE_TRACE builds: entries written to trace[]
    unsigned int pad[61];
    unsigned short team_start[kMaxBatch + 2];  // variable teams: team i = CTAs [start[i], start[i+1])
    double partial[kMaxCtas * kMaxDots];
    unsigned long long trace[kTraceEntries];   // (code << 48) | globaltimer ns
};

template <typename W> struct Prec;
template <> struct Prec<double> {
    FDE_D static const cx<double>* tw(const Inst& I) { return I.tw64; }
    FDE_D static const cx<double>* lam(const AxisData& a) { return a.lam64; }
    FDE_D static const double* phi(const AxisData& a) { return a.phi64; }
    FDE_D static const double* dp(const Inst& I) { return I.dp64; }
    FDE_D static const double* dm(const Inst& I) { return I.dm64; }
    FDE_D static const double* ep(const Inst& I) { return I.ep64; }
    FDE_D static const double* em(const Inst& I) { return I.em64; }
    FDE_D static const double* dinv(const Inst& I) { return I.dinv64; }
    FDE_D static const double* tri(const Inst& I) { return I.tri64; }
    FDE_D static cx<double>* split(const Inst& I) { return reinterpret_cast<cx<double>*>(I.split64); }
};
template <> struct Prec<float> {
    FDE_D static const cx<float>* tw(const Inst& I) { return I.tw32; }
    FDE_D static const cx<float>* lam(const AxisData& a) { return a.lam32; }
    FDE_D static const float* phi(const AxisData& a) { return a.phi32; }
    FDE_D static const float* dp(const Inst& I) { return I.dp32; }
    FDE_D static const float* dm(const Inst& I) { return I.dm32; }
    FDE_D static const float* ep(const Inst& I) { return I.ep32; }
    FDE_D static const float* em(const Inst& I) { return I.em32; }
    FDE_D static const float* dinv(const Inst& I) { return I.dinv32; }
    FDE_D static const float* tri(const Inst& I) { return I.tri32; }
    FDE_D static cx<float>* split(const Inst& I) { return reinterpret_cast<cx<float>*>(I.split32); }
};

}  // namespace fde
