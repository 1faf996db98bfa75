// Spectral-bound estimates for the expansion (Sec. II-C: the polynomial
// expansions need estimates eps_1, eps_N of the spectral bounds, and the
// number of products grows with the width they span).
//
// Gershgorin discs always contain the spectrum but, for a dense rotated Hp,
// span ~20-50x its true width, which costs SP2 about 2 log2 of that ratio in
// extra products (and the finite-temperature recursion extra doublings).
// Here kLanczosSteps steps of the Lanczos recurrence (FP32 vectors and
// products, FP64 sums), from a fixed
// pseudo-random unit vector, give Ritz values theta_min, theta_max inside the
// spectrum; the estimate is
//     [theta_min - |beta_k s_min|, theta_max + |beta_k s_max|],
// widened by the residuals of the extreme Ritz pairs (s the unit eigenvector
// of the tridiagonal T) and clipped to the Gershgorin interval.
//
// An estimate is not a bound, so it is certified before use (k_check_bounds):
// with X0 = (hi I - Hp)/(hi - lo), kCheckSteps logistic steps
// X <- 4 X (I - X) give X_3 = (I - T_8(A))/2, T_8 the Chebyshev polynomial and
// A = (2 Hp - (hi + lo) I)/(hi - lo).  |T_8| <= 1 on [-1, 1] and
// T_8(a) = cosh(8 arccosh |a|) outside, so every eigenvalue a of A satisfies
// (cosh(8 arccosh |a|) - 1)/2 <= ||X_3||_F, i.e.
//     |a| <= cosh(arccosh(1 + 2 ||X_3||_F) / 8),
// and the interval widened by that factor contains the spectrum.  Eigenvalues
// inside the estimate keep X_3 in [0, 1] (||X_3||_F <= sqrt(n): at most a
// ~25% widening); one that the estimate missed grows X_3 and widens the
// bound just enough to take it in.
//
// No reorthogonalisation: loss of orthogonality only repeats converged Ritz
// values, which cannot move the extreme ones outward.
#include <cfloat>

#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {

namespace {

// SplitMix64 finaliser: a fixed, well-mixed 64-bit value per index
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double block_sum_1024(double v, double *sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) sh[t] += sh[t + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// number of eigenvalues of the tridiagonal (a, b) below x (Sturm sequence),
// in FP32 with the squared couplings b2[i] = b[i]^2 (GB300 runs FP64 at 1/64
// of the FP32 rate; the estimate needs no more than FP32 precision, since the
// certificate that follows decides the bounds)
__device__ int sturm_count_f(const float *a, const float *b2, int k, float x) {
    int c = 0;
    float q = a[0] - x;
    if (q < 0.0f) ++c;
    for (int i = 1; i < k; ++i) {
        if (q == 0.0f) q = 1e-30f;
        q = a[i] - x - b2[i] / q;
        if (q < 0.0f) ++c;
    }
    return c;
}

// eigenvalue number `idx` (0-based, ascending) of T in [lo, hi] by 32-point
// multisection over the warp (every lane calls it): each round lane l counts
// the eigenvalues below lo + (hi - lo)(l + 1)/33, and the interval shrinks to
// the two neighbouring points that bracket eigenvalue idx (33x per round),
// down to FP32 resolution.
__device__ double tri_eig(const float *a, const float *b2, int k, int idx, double lo, double hi) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < 8; ++r) {
        const double w = hi - lo;
        if (!(w > 3e-7 * fmax(fabs(lo), fabs(hi)))) break;
        const double x = lo + w * static_cast<double>(lane + 1) / 33.0;
        const unsigned above = __ballot_sync(0xffffffffu, sturm_count_f(a, b2, k, static_cast<float>(x)) > idx);
        const int f = above ? __ffs(above) - 1 : 32;  // first point above the eigenvalue
        const double nlo = lo + w * static_cast<double>(f) / 33.0;
        const double nhi = (f < 32) ? lo + w * static_cast<double>(f + 1) / 33.0 : hi;
        lo = nlo;
        hi = nhi;
    }
    return 0.5 * (lo + hi);
}

// |last component| of the unit eigenvector of T for eigenvalue th (forward
// three-term recurrence, rescaled to stay finite)
__device__ double tri_last_comp(const double *a, const double *b, int k, double th) {
    double s_prev = 0.0, s = 1.0, norm2 = 1.0;
    for (int i = 0; i + 1 < k; ++i) {
        // (a_i - th) s_i + b_i s_{i-1} + b_{i+1} s_{i+1} = 0
        const double bn = b[i + 1];
        const double s_next = (bn != 0.0) ? -((a[i] - th) * s + b[i] * s_prev) / bn : 0.0;
        s_prev = s;
        s = s_next;
        norm2 += s * s;
        if (norm2 > 1e200) {
            const double r = 1e-100;
            s *= r;
            s_prev *= r;
            norm2 *= r * r;
        }
    }
    return fabs(s) / sqrt(norm2);
}

}  // namespace

// The recurrence runs in FP32 (vectors, H entries, products) with FP64 sums:
// the estimate needs no more (the certificate decides the bounds), and GB300
// runs FP64 arithmetic at 1/64 of the FP32 rate.

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number k of a cooperative launch: complete once all nb blocks
// arrived, i.e. the arrival counter (zeroed before the launch) reaches
// (k + 1) nb.  The wait is bounded: when it runs out the block records
// kErrTimeoutGrid and every caller returns false (the blocks still running
// give up at their own next barrier).
__device__ bool grid_barrier(unsigned *cnt, unsigned k, unsigned nb, DevCtl *ctl, int *flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(cnt, 1u);
        const unsigned target = (k + 1u) * nb;
        bool ok = true;
        if (ld_acquire_u32(cnt) < target) {
            const uint64_t lim = ctl->wait_ns, t0 = globaltimer();
            while (ld_acquire_u32(cnt) < target) {
                if (globaltimer() - t0 > lim) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (!ok) atomicCAS(&ctl->err, 0, kErrTimeoutGrid);
        __threadfence();
        *flag = ok ? 1 : 0;
    }
    __syncthreads();
    return *flag != 0;
}

// v = fixed pseudo-random unit vector, v_prev = 0 (the whole block)
__device__ void lz_start(const MmaProb &pr, double *sh) {
    SolveState *st = pr.st;
    if (!st->lz_on) return;
    const int n = pr.n;
    float *vp = pr.lzv, *v = pr.lzv + n;
    double ss = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float x = static_cast<float>(static_cast<double>(mix64(0xF00Dull + static_cast<uint64_t>(i)) >> 11) *
                                           (2.0 / 9007199254740992.0) - 1.0);  // uniform in [-1, 1)
        v[i] = x;
        vp[i] = 0.0f;
        ss += static_cast<double>(x) * x;
    }
    const double nrm = sqrt(block_sum_1024(ss, sh));
    const float inv = nrm > 0.0 ? static_cast<float>(1.0 / nrm) : 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] *= inv;
    if (threadIdx.x == 0) {
        st->lz_k = 0;
        st->lz_b[0] = 0.0;
    }
}

// This block's share of w = H v: rows blockIdx.x * kWarps + warp, stepping
// by the grid's warps, one warp per row.  H is read from its FP32 copy in the
// problem's FP32 master (written by k_bounds_rows; rows 16-byte aligned, ld a
// multiple of 4) as 16-byte quadruples, four per lane in flight.  v comes
// from shared memory when `vs` holds it, else from L2 (ld.cg: another block
// wrote it since this launch began, so L1 may hold a stale copy).  The
// block's partial of w . v goes to its partial slot.
template <bool kStaged>
__device__ void lz_matvec(const MmaProb &pr, const float *vs, double *red) {
    constexpr int kWarps = kLzThreads / 32;
    const int n = pr.n;
    const float *v = kStaged ? vs : pr.lzv + n;
    float *w = pr.lzv + 2 * static_cast<size_t>(n);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    auto vat = [&](int i) { return kStaged ? v[i] : __ldcg(v + i); };
    double part = 0.0;
    for (int row = blockIdx.x * kWarps + wid; row < n; row += gridDim.x * kWarps) {
        const float *h = pr.Y + static_cast<size_t>(row) * pr.ldy;
        const int m = n >> 2;  // 16-byte quadruples
        const float4 *h4 = reinterpret_cast<const float4 *>(h);
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        int k = lane;
        auto dot4 = [&](const float4 a, int q, float acc) {
            return fmaf(a.x, vat(4 * q), fmaf(a.y, vat(4 * q + 1), fmaf(a.z, vat(4 * q + 2), fmaf(a.w, vat(4 * q + 3), acc))));
        };
        for (; k + 96 < m; k += 128) {
            const float4 a0 = h4[k], a1 = h4[k + 32], a2 = h4[k + 64], a3 = h4[k + 96];
            s0 = dot4(a0, k, s0);
            s1 = dot4(a1, k + 32, s1);
            s2 = dot4(a2, k + 64, s2);
            s3 = dot4(a3, k + 96, s3);
        }
        for (; k < m; k += 32) s0 = dot4(h4[k], k, s0);
        for (int jj = 4 * m + lane; jj < n; jj += 32) s1 = fmaf(h[jj], vat(jj), s1);
        const double s = warp_sum(static_cast<double>((s0 + s1) + (s2 + s3)));
        if (lane == 0) {
            w[row] = static_cast<float>(s);
            part += s * static_cast<double>(vat(row));
        }
    }
    if (lane == 0) red[wid] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < kWarps; ++q) a += red[q];
        pr.part[static_cast<size_t>(blockIdx.x) * kPartStride] = a;
    }
    __syncthreads();
}

// alpha_j = w . v (the blocks' partials, in block order); w' = w - alpha_j v
// - beta_j v_prev; beta_{j+1} = ||w'||; v_prev <- v, v <- w' / beta_{j+1}
// (the whole block; everything another block wrote is read through L2)
__device__ void lz_update(const MmaProb &pr, int j, double *sh) {
    SolveState *st = pr.st;
    const int n = pr.n;
    float *vp = pr.lzv, *v = pr.lzv + n, *w = pr.lzv + 2 * static_cast<size_t>(n);
    double a = 0.0;
    for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += blockDim.x)
        a += __ldcg(pr.part + static_cast<size_t>(b) * kPartStride);
    const double alpha = block_sum_1024(a, sh);
    const double beta = st->lz_b[j];
    const float af = static_cast<float>(alpha), bf = static_cast<float>(beta);
    float ssf = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float x = fmaf(-af, v[i], fmaf(-bf, vp[i], __ldcg(w + i)));
        w[i] = x;
        ssf = fmaf(x, x, ssf);
    }
    const double bn = sqrt(block_sum_1024(static_cast<double>(ssf), sh));
    const bool stop = !(bn > 1e-6 * fmax(fabs(alpha), 1e-300));  // invariant subspace (to FP32 accuracy)
    const float inv = stop ? 0.0f : static_cast<float>(1.0 / bn);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        vp[i] = v[i];
        v[i] = w[i] * inv;
    }
    if (threadIdx.x == 0) {
        st->lz_a[j] = alpha;
        st->lz_b[j + 1] = stop ? 0.0 : bn;
        st->lz_k = stop ? -(j + 1) : j + 1;  // negative: stopped after |lz_k| steps
    }
}

// bounds from the tridiagonal, then the X0 preparation (warp 0 of the block)
__device__ void lz_finish(const MmaProb &pr, double narrow) {
    SolveState *st = pr.st;
    const int lane = threadIdx.x & 31;
    const int k = st->lz_k < 0 ? -st->lz_k : st->lz_k;
    const double glo = st->gersh_lo, ghi = st->gersh_hi;
    __shared__ double a[kLanczosSteps], b[kLanczosSteps + 1];  // b[i] couples i-1 and i, b[k] the residual
    __shared__ float af[kLanczosSteps], b2f[kLanczosSteps + 1];
    if (lane < kLanczosSteps) {
        a[lane] = st->lz_a[lane];
        af[lane] = static_cast<float>(a[lane]);
    }
    if (lane <= kLanczosSteps) {
        b[lane] = st->lz_b[lane];
        b2f[lane] = static_cast<float>(b[lane] * b[lane]);
    }
    __syncwarp();
    double lo = glo, hi = ghi;
    if (k >= 2) {
        const double tmin = tri_eig(af, b2f, k, 0, glo, ghi);
        const double tmax = tri_eig(af, b2f, k, k - 1, glo, ghi);
        const double rmin = b[k] * tri_last_comp(a, b, k, tmin);
        const double rmax = b[k] * tri_last_comp(a, b, k, tmax);
        lo = fmax(glo, tmin - rmin);
        hi = fmin(ghi, tmax + rmax);
        if (!(hi > lo)) {
            lo = glo;
            hi = ghi;
        }
    }
    __syncwarp();
    if (lane != 0) return;
    if (narrow < 1.0) {
        const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo) * narrow;
        lo = mid - half;
        hi = mid + half;
    }
    // X0 on the estimate, for the certificate steps (k_control issues them)
    st->lz_lo = lo;
    st->lz_hi = hi;
    st->chk_left = kCheckSteps;
    setup_from_bounds(pr, st, lo, hi);
}

}  // namespace

// The whole estimate in one cooperative launch (see fe_kernels.cuh).  Block b
// starts, updates and finishes the problems b, b + grid, ...; every block
// takes part in every product.  Each product and each update ends at a grid
// barrier; a problem whose recurrence stopped (lz_k < 0, written by its
// updating block before the barrier) is skipped from then on.
__global__ void __launch_bounds__(kLzThreads, 2)
    k_lanczos_run(const MmaProb *probs, int k0, int m, int vcap, double narrow, DevCtl *ctl, unsigned *bar) {
    extern __shared__ float vs[];  // v of the problem in hand, when n <= vcap
    __shared__ double sh[kLzThreads];
    __shared__ int flag;
    const unsigned nb = gridDim.x;
    unsigned nbar = 0;
    for (int q = blockIdx.x; q < m; q += nb) lz_start(probs[k0 + q], sh);
    if (!grid_barrier(bar, nbar++, nb, ctl, &flag)) return;
    for (int j = 0; j < kLanczosSteps; ++j) {
        for (int q = 0; q < m; ++q) {
            const MmaProb &pr = probs[k0 + q];
            const SolveState *st = pr.st;
            if (!st->lz_on || *reinterpret_cast<const volatile int *>(&st->lz_k) < 0) continue;
            const int n = pr.n;
            if (n <= vcap) {
                for (int i = threadIdx.x; i < n; i += blockDim.x) vs[i] = __ldcg(pr.lzv + n + i);
                __syncthreads();
                lz_matvec<true>(pr, vs, sh);
            } else {
                lz_matvec<false>(pr, vs, sh);
            }
        }
        if (!grid_barrier(bar, nbar++, nb, ctl, &flag)) return;
        for (int q = blockIdx.x; q < m; q += nb) {
            const MmaProb &pr = probs[k0 + q];
            if (pr.st->lz_on && pr.st->lz_k >= 0) lz_update(pr, j, sh);
            __syncthreads();
        }
        if (!grid_barrier(bar, nbar++, nb, ctl, &flag)) return;
    }
    if (threadIdx.x < 32)
        for (int q = blockIdx.x; q < m; q += nb)
            if (probs[k0 + q].st->lz_on) lz_finish(probs[k0 + q], narrow);
}

// Certified bounds from the check steps, then the X0 preparation (one thread
// per problem, blockIdx.x)
__global__ void k_check_bounds(const MmaProb *probs, int k0) {
    const MmaProb &pr = probs[k0 + blockIdx.x];
    SolveState *st = pr.st;
    if (threadIdx.x != 0 || !st->lz_on) return;
    const double mid = 0.5 * (st->lz_lo + st->lz_hi), half = 0.5 * (st->lz_hi - st->lz_lo);
    const double a = st->chk_amax;
    double lo = st->gersh_lo, hi = st->gersh_hi;
    if (a < 1e300 && half > 0.0) {  // NaN and overflow keep the Gershgorin interval
        lo = fmax(lo, mid - half * a);
        hi = fmin(hi, mid + half * a);
    }
    st->chk = 0;
    st->chk_left = 0;
    st->kind = kNone;
    setup_from_bounds(pr, st, lo, hi);
}

}  // namespace fe
