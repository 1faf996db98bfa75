// FP64-accurate SP2 step (Sec. II-B1 Eq. (1)) on the upper-triangle 64x64
// tiles of X^2, for the final polishing products of the mixed schedule (Sec.
// III-A: the last iterations run in FP64) and for every product of the plain
// FP64 schedule.  (X^2)_ij = sum_k X_ik X_jk since X is symmetric.  The
// epilogue writes X' = X^2 or 2X - X^2 to the other FP64 buffer (and its
// mirror) and per-tile partials: tr X', ||X'||_F^2 and ||X^2 - X||_F^2.
//
// Two arithmetics, chosen per problem by the control kernel:
//   kFp64  native FP64 fused multiply-adds (the plain FP64 schedule);
//   kDf    double-float: every operand is split into an FP32 pair
//          x = x_h + x_l, each product x_h y_h is made exact with an FMA
//          (TwoProduct), the cross terms x_h y_l + x_l y_h are added in
//          FP32, and the running sum is a pair renormalised with the
//          error-free TwoSum of Knuth.  About 2^-45 relative accuracy at
//          roughly 7x the speed of GB300's FP64 units.
#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {

namespace {
constexpr int kBK = 16;

struct XSrc {
    const double *X;  // FP64 iterate, or null when reading c I + Y
    const float *Y;
    double c;
    int ld;
    int n;
    __device__ __forceinline__ double at(int i, int k) const {
        if (i >= n || k >= n) return 0.0;
        if (X) return X[static_cast<long long>(i) * ld + k];
        return static_cast<double>(Y[static_cast<long long>(i) * ld + k]) + (i == k ? c : 0.0);
    }
};

// (hi, lo) += a * b for a = (ah, al), b = (bh, bl), all FP32.
__device__ __forceinline__ void df_fma(float &hi, float &lo, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);        // exact: ah bh = p + e
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float s = __fadd_rn(hi, p);       // TwoSum(hi, p) -> (s, t)
    const float v = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, e));
}

struct Partials {
    double tr = 0.0, s2 = 0.0, id = 0.0;
};

// Epilogue shared by both arithmetics: P = (X^2)_ij for this thread's 4x4.
__device__ __forceinline__ void step_epilogue(const MmaProb &pr, const SolveState *st,
                                              const XSrc &src, int i0, int j0, int tx, int ty,
                                              const double (&P)[4][4], Partials &pa) {
    double *Xo = pr.Xd[st->xcur ^ 1];  // the control kernel flips xcur afterwards
    const int sq = st->sq;
    const int chk = st->chk;  // bound-certificate step: X' = 4 X (I - X)
    const double gamma = st->gamma;
    const int n = src.n;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty + 16 * r;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx + 16 * q;
            if (i >= n || j >= n || j < i) continue;
            const double xo = src.at(i, j);
            // SP2 branch plus the trace correction gamma (X - X^2), which
            // commutes with Hp and moves each eigenvalue by gamma x (1 - x)
            const double xn = chk ? 4.0 * (xo - P[r][q])
                                  : (sq ? P[r][q] : 2.0 * xo - P[r][q]) + gamma * (xo - P[r][q]);
            Xo[static_cast<long long>(i) * pr.ldx + j] = xn;
            const double dd = P[r][q] - xo;
            if (j != i) {
                Xo[static_cast<long long>(j) * pr.ldx + i] = xn;
                pa.s2 += 2.0 * xn * xn;
                pa.id += 2.0 * dd * dd;
            } else {
                pa.tr += xn;
                pa.s2 += xn * xn;
                pa.id += dd * dd;
            }
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(256) k_fp64_step(const MmaProb *probs, const Tile64 *tiles,
                                                   int ntiles) {
    __shared__ double sA[kBK][kTile64 + 1];
    __shared__ double sB[kBK][kTile64 + 1];
    __shared__ float fAh[kBK][kTile64 + 4], fAl[kBK][kTile64 + 4];
    __shared__ float fBh[kBK][kTile64 + 4], fBl[kBK][kTile64 + 4];
    __shared__ double red[3][8];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile64 te = tiles[t];
        const MmaProb &pr = probs[te.prob];
        const SolveState *st = pr.st;
        const int kind = *reinterpret_cast<const volatile int *>(&st->kind);
        if (kind != kFp64 && kind != kDf) continue;
        const int n = pr.n;
        XSrc src;
        if (st->x_fp64) {
            src.X = pr.Xd[st->xcur];
            src.Y = nullptr;
            src.ld = pr.ldx;
        } else {
            src.X = nullptr;
            src.Y = pr.Y;
            src.ld = pr.ldy;
        }
        src.c = st->c;
        src.n = n;
        const int i0 = te.I * kTile64, j0 = te.J * kTile64;
        double P[4][4];
        if (kind == kFp64) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) P[r][q] = 0.0;
            for (int k0 = 0; k0 < n; k0 += kBK) {
                for (int e = threadIdx.x; e < kTile64 * kBK; e += 256) {
                    const int r = e / kBK, kk = e % kBK;
                    sA[kk][r] = src.at(i0 + r, k0 + kk);
                    sB[kk][r] = src.at(j0 + r, k0 + kk);
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < kBK; ++kk) {
                    double a[4], b[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) a[r] = sA[kk][ty + 16 * r];
#pragma unroll
                    for (int q = 0; q < 4; ++q) b[q] = sB[kk][tx + 16 * q];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int q = 0; q < 4; ++q) P[r][q] = fma(a[r], b[q], P[r][q]);
                }
                __syncthreads();
            }
        } else {
            float ch[4][4], cl[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) { ch[r][q] = 0.0f; cl[r][q] = 0.0f; }
            for (int k0 = 0; k0 < n; k0 += kBK) {
                for (int e = threadIdx.x; e < kTile64 * kBK; e += 256) {
                    const int r = e / kBK, kk = e % kBK;
                    const double a = src.at(i0 + r, k0 + kk);
                    const double b = src.at(j0 + r, k0 + kk);
                    const float ah = __double2float_rn(a), bh = __double2float_rn(b);
                    fAh[kk][r] = ah;
                    fAl[kk][r] = __double2float_rn(a - static_cast<double>(ah));
                    fBh[kk][r] = bh;
                    fBl[kk][r] = __double2float_rn(b - static_cast<double>(bh));
                }
                __syncthreads();
#pragma unroll 4
                for (int kk = 0; kk < kBK; ++kk) {
                    float ah[4], al[4], bh[4], bl[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) { ah[r] = fAh[kk][ty + 16 * r]; al[r] = fAl[kk][ty + 16 * r]; }
#pragma unroll
                    for (int q = 0; q < 4; ++q) { bh[q] = fBh[kk][tx + 16 * q]; bl[q] = fBl[kk][tx + 16 * q]; }
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int q = 0; q < 4; ++q) df_fma(ch[r][q], cl[r][q], ah[r], al[r], bh[q], bl[q]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    P[r][q] = static_cast<double>(ch[r][q]) + static_cast<double>(cl[r][q]);
        }

        Partials pa;
        step_epilogue(pr, st, src, i0, j0, tx, ty, P, pa);
        double tr = warp_sum(pa.tr), s2 = warp_sum(pa.s2), id = warp_sum(pa.id);
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) { red[0][wid] = tr; red[1][wid] = s2; red[2][wid] = id; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0, c = 0;
            for (int w = 0; w < 8; ++w) { a += red[0][w]; b += red[1][w]; c += red[2][w]; }
            double *slot = pr.part + static_cast<size_t>(te.slot) * kPartStride;
            slot[0] = a;
            slot[1] = b;
            slot[2] = 0.0;
            slot[3] = c;
        }
        __syncthreads();
    }
}

}  // namespace fe
