// FP64 SP2 step (Sec. II-B1 Eq. (1)) on the upper-triangle 64x64 tiles of
// X^2, used for the final polishing products of the mixed schedule (Sec.
// III-A: the last iterations run in FP64) and for every product of the plain
// FP64 schedule.  (X^2)_ij = sum_k X_ik X_jk since X is symmetric.  The
// epilogue writes X' = X^2 or 2X - X^2 to the other FP64 buffer (and its
// mirror) and per-tile partials: tr X', ||X'||_F^2 and ||X^2 - X||_F^2.
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
}  // namespace

__global__ void __launch_bounds__(256) k_fp64_step(const MmaProb *probs, const Tile64 *tiles,
                                                   int ntiles) {
    __shared__ double sA[kBK][kTile64 + 1];
    __shared__ double sB[kBK][kTile64 + 1];
    __shared__ double red[3][8];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile64 te = tiles[t];
        const MmaProb &pr = probs[te.prob];
        const SolveState *st = pr.st;
        if (*reinterpret_cast<const volatile int *>(&st->kind) != kFp64) continue;
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
        double acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = 0.0;

        for (int k0 = 0; k0 < n; k0 += kBK) {
            // 64 rows x 16 k of each panel: 1024 values, 4 per thread
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
                    for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
            }
            __syncthreads();
        }

        // the result always goes to the other buffer; the control kernel flips xcur
        double *Xo = pr.Xd[st->xcur ^ 1];
        const int sq = st->sq;
        double tr = 0.0, s2 = 0.0, id = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + ty + 16 * r;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + tx + 16 * q;
                if (i >= n || j >= n || j < i) continue;
                const double P = acc[r][q];
                const double xo = src.at(i, j);
                const double xn = sq ? P : 2.0 * xo - P;
                Xo[static_cast<long long>(i) * pr.ldx + j] = xn;
                const double dd = P - xo;
                if (j != i) {
                    Xo[static_cast<long long>(j) * pr.ldx + i] = xn;
                    s2 += 2.0 * xn * xn;
                    id += 2.0 * dd * dd;
                } else {
                    tr += xn;
                    s2 += xn * xn;
                    id += dd * dd;
                }
            }
        }
        tr = warp_sum(tr);
        s2 = warp_sum(s2);
        id = warp_sum(id);
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
