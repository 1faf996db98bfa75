// Bandwidth-bound kernels around the expansion loop:
//   * Gershgorin bounds of Hp (Sec. II-C: the expansion needs spectral bounds
//     eps_1, eps_N; taken as Gershgorin discs), with tr Hp and a NaN/Inf scan.
//   * X0 = (eps_max I - Hp) / (eps_max - eps_min) (spectrum in [0, 1], occupied
//     states toward 1), stored as X0 = c0 I + Y0 with c0 = tr X0 / n, plus the
//     first FP16 slices and per-block partials of tr Y0 and ||Y0||_F^2.
//   * Output: D = X written to the caller's layout, and the FP64 band energy
//     tr(Hp D) = sum_ij Hp_ij D_ij (Sec. III-C) and tr D.
// Every reduction is a fixed-order tree, so results are bitwise reproducible.
#include <cfloat>
#include <type_traits>

#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {

__global__ void k_bounds_rows(const MmaProb *probs, int prob, RowInfo *rowinfo, int *bad) {
    const MmaProb &pr = probs[prob];
    const int warps_per_block = blockDim.x >> 5;
    const int row = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= pr.n) return;
    const double *h = pr.H + static_cast<long long>(row) * pr.ldh;
    // |h| and the NaN/Inf test work on the bit patterns (for non-negative
    // doubles their order as integers is their order as values): the one
    // FP64 operation per element is the row sum (GB300 runs FP64 at 1/64 of
    // the FP32 rate)
    constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kExp = 0x7FF0000000000000ull;
    double s = 0.0;
    unsigned long long mxb = 0, nonfin = 0;
    // four loads per lane in flight: the 128 to 2048 rows an SM holds must
    // keep enough bytes outstanding to stream Hp at HBM speed
    // The row also goes to the FP32 master as an FP32 copy of Hp for the
    // Lanczos matvecs (read 12 times; at 4n^2 bytes it stays in L2 up to
    // n ~ 5600); the master is free until X0 is written.
    float *yrow = pr.Y + static_cast<long long>(row) * pr.ldy;
    int j = lane;
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (; j + 96 < pr.n; j += 128) {
        const double h0 = h[j], h1 = h[j + 32], h2 = h[j + 64], h3 = h[j + 96];
        yrow[j] = f64_to_f32_rn(h0);
        yrow[j + 32] = f64_to_f32_rn(h1);
        yrow[j + 64] = f64_to_f32_rn(h2);
        yrow[j + 96] = f64_to_f32_rn(h3);
        const unsigned long long b0 = static_cast<unsigned long long>(__double_as_longlong(h0)) & kAbs;
        const unsigned long long b1 = static_cast<unsigned long long>(__double_as_longlong(h1)) & kAbs;
        const unsigned long long b2 = static_cast<unsigned long long>(__double_as_longlong(h2)) & kAbs;
        const unsigned long long b3 = static_cast<unsigned long long>(__double_as_longlong(h3)) & kAbs;
        nonfin |= ((b0 & kExp) == kExp) | ((b1 & kExp) == kExp) | ((b2 & kExp) == kExp) | ((b3 & kExp) == kExp);
        s += __longlong_as_double(static_cast<long long>(b0));
        s1 += __longlong_as_double(static_cast<long long>(b1));
        s2 += __longlong_as_double(static_cast<long long>(b2));
        s3 += __longlong_as_double(static_cast<long long>(b3));
        mxb = max(max(mxb, b0), max(b1, max(b2, b3)));
    }
    for (; j < pr.n; j += 32) {
        const double h0 = h[j];
        yrow[j] = f64_to_f32_rn(h0);
        const unsigned long long b0 = static_cast<unsigned long long>(__double_as_longlong(h0)) & kAbs;
        nonfin |= ((b0 & kExp) == kExp);
        s += __longlong_as_double(static_cast<long long>(b0));
        mxb = max(mxb, b0);
    }
    s = warp_sum((s + s1) + (s2 + s3));
    for (int o = 16; o > 0; o >>= 1) mxb = max(mxb, __shfl_xor_sync(0xffffffffu, mxb, o));
    const double mx = __longlong_as_double(static_cast<long long>(mxb));
    int nonfinite = nonfin ? 1 : 0;
    nonfinite = __any_sync(0xffffffffu, nonfinite);
    if (lane == 0) {
        const double d = h[row];
        const double r = s - fabs(d);
        rowinfo[row] = RowInfo{d - r, d + r, d, mx};
        if (nonfinite) atomicExch(bad, 1);
    }
}

__global__ void k_bounds_reduce(const MmaProb *probs, int prob, const RowInfo *rowinfo,
                                const int *bad) {
    const MmaProb &pr = probs[prob];
    SolveState *st = pr.st;
    __shared__ double s_lo[1024], s_hi[1024], s_tr[1024], s_mx[1024];
    const int t = threadIdx.x;
    double lo = DBL_MAX, hi = -DBL_MAX, tr = 0.0, mx = 0.0;
    for (int i = t; i < pr.n; i += blockDim.x) {
        const RowInfo r = rowinfo[i];
        lo = fmin(lo, r.lo);
        hi = fmax(hi, r.hi);
        tr += r.diag;
        mx = fmax(mx, r.maxabs);
    }
    s_lo[t] = lo; s_hi[t] = hi; s_tr[t] = tr; s_mx[t] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            s_lo[t] = fmin(s_lo[t], s_lo[t + o]);
            s_hi[t] = fmax(s_hi[t], s_hi[t + o]);
            s_tr[t] += s_tr[t + o];
            s_mx[t] = fmax(s_mx[t], s_mx[t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        st->gersh_lo = s_lo[0];
        st->gersh_hi = s_hi[0];
        st->trH = s_tr[0];
        st->hmax = s_mx[0];
        st->bad_input = *bad;
        if (!st->lz_on) setup_from_bounds(pr, st, s_lo[0], s_hi[0]);
    }
}

// Y0 = X0 - c0 I with X0 = (eps_max I - Hp) / w; FP32 master + FP16 slices of s0 Y0.
// For the all-FP64 schedule X0 itself goes to Xd[0] in FP64.
__global__ void __launch_bounds__(256, 4) k_init_x0(const MmaProb *probs, int prob) {
    const MmaProb &pr = probs[prob];
    SolveState *st = pr.st;
    const int n = pr.n;
    double w = st->emax - st->emin;
    if (!(w > 0.0)) w = 1.0;
    const double inv_w = 1.0 / w;
    const double dshift = st->emax * inv_w - st->c;  // diagonal of Y0 gets +dshift
    const float s0 = st->s_cur;
    const bool fp64 = (st->prec == kPrecFp64);
    // the certificate steps start from X0 in the zero-temperature form
    const bool fermi = (st->method == kMethodFermi) && st->chk_left == 0;
    const double hb0 = 0.5 * st->beta0, mu0 = st->mu_t;
    const float sz = st->scl[kMatZ];
    // FP32 arithmetic off the diagonal (GB300 runs FP64 at 1/64 of the FP32
    // rate, and the FP32 result is what is stored); each thread's squares are
    // summed in FP32 over its columns of one row (at most n / blockDim terms),
    // then in FP64 across rows
    const float inv_wf = static_cast<float>(inv_w), hb0f = static_cast<float>(hb0);
    // everything the loop needs, read once: the stores below could alias the
    // problem table as far as the compiler knows, which would reload these
    // after every store
    const MatSlot &msl = pr.mats[fermi ? kMatZ : kMatY0];
    float *const mbase = msl.master;
    __half *const s0base = msl.sl[0];
    __half *const s1base = msl.sl[1];
    const float sc = fermi ? sz : s0;
    const double *const hbase = pr.H;
    const long long ldh = pr.ldh, ldy = pr.ldy, lds = pr.lds, ldx = pr.ldx;
    double *const xbase = pr.Xd[0];
    double *const dgz = pr.dg[kMatZ];
    float *const dgzf = pr.dgf[kMatZ];
    const double emax = st->emax;
    double tr = 0.0, sq = 0.0;
    // one warp per row (warp w of the grid takes rows w, w + warps, ...); lane
    // l the column pairs (2l, 2l + 1), (2l + 64, ...), ...: 16-byte loads of Hp
    // where its row is aligned, 8-byte FP32 and 4-byte FP16 stores (ldy and
    // lds are even).  Four column pairs per lane are loaded before any is used;
    // with every row of n <= 4864 in flight at once (kInitBlocks blocks of 8
    // warps), the bytes outstanding approach the HBM rate.
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    // one instantiation of the row loop per form (0: zero temperature, 1:
    // finite temperature, 2: the FP64 schedule), so each keeps only its own
    // registers live
    auto rows = [&](auto form) {
        constexpr int kForm = decltype(form)::value;
        for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
            float sqr = 0.0f;
            double sqd = 0.0;
            const double *hrow = hbase + static_cast<long long>(i) * ldh;
            const bool h16 = (reinterpret_cast<uintptr_t>(hrow) & 15u) == 0;
            float *const mrow = mbase + static_cast<long long>(i) * ldy;
            __half *const s0row = s0base + static_cast<long long>(i) * lds;
            __half *const s1row = s1base + static_cast<long long>(i) * lds;
            auto body = [&](int j, double h0, double h1) {
                const bool two = j + 1 < n;
                if constexpr (kForm == 2) {
                    double *xr = xbase + static_cast<long long>(i) * ldx;
                    const double x0 = ((i == j) ? emax - h0 : -h0) * inv_w;
                    xr[j] = x0;
                    if (i == j) tr += x0;
                    sqd += x0 * x0;
                    if (two) {
                        const double x1 = ((i == j + 1) ? emax - h1 : -h1) * inv_w;
                        xr[j + 1] = x1;
                        if (i == j + 1) tr += x1;
                        sqd += x1 * x1;
                    }
                    return;
                }
                // FP32 only here (GB300 runs FP64 at 1/64 of the FP32 rate, and an
                // FP64 expression guarded by i == j is still evaluated for every
                // element); the diagonal entry is written as 0 and set after the
                // row's loop by the lane that owns it
                const float f = (kForm == 1) ? hb0f : -inv_wf;
                const float y0 = (i == j) ? 0.0f : f * f64_to_f32_rn(h0);
                const float y1 = (i == j + 1 || !two) ? 0.0f : f * f64_to_f32_rn(h1);
                const float ys0 = y0 * sc, ys1 = y1 * sc;
                const __half a0 = __float2half_rn(ys0), a1 = __float2half_rn(ys1);
                const __half b0 = __float2half_rn(ys0 - __half2float(a0)), b1 = __float2half_rn(ys1 - __half2float(a1));
                if (two) {
                    *reinterpret_cast<float2 *>(mrow + j) = make_float2(y0, y1);
                    *reinterpret_cast<__half2 *>(s0row + j) = __halves2half2(a0, a1);
                    *reinterpret_cast<__half2 *>(s1row + j) = __halves2half2(b0, b1);
                } else {
                    mrow[j] = y0;
                    s0row[j] = a0;
                    s1row[j] = b0;
                }
                sqr = fmaf(y0, y0, fmaf(y1, y1, sqr));
            };
            for (int jb = 2 * lane; jb < n; jb += 4 * 64) {
                double hx[4], hy[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = jb + q * 64;
                    hx[q] = 0.0;
                    hy[q] = 0.0;
                    if (j < n) {
                        if (j + 1 < n && h16) {
                            const double2 hv = *reinterpret_cast<const double2 *>(hrow + j);
                            hx[q] = hv.x;
                            hy[q] = hv.y;
                        } else {
                            hx[q] = hrow[j];
                            if (j + 1 < n) hy[q] = hrow[j + 1];
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = jb + q * 64;
                    if (j < n) body(j, hx[q], hy[q]);
                }
            }
            if (kForm != 2 && lane == ((i & 63) >> 1)) {
                // the diagonal entry, in FP64: finite temperature keeps it in d_Z
                // (the small part stays 0 there), zero temperature in Y0
                const double hd = hrow[i];
                if (kForm == 1) {
                    const double dv = hb0 * (hd - mu0);
                    dgz[i] = dv;
                    dgzf[i] = static_cast<float>(dv);
                    tr += dv;
                    sqd += dv * dv;
                } else {
                    const float yd = static_cast<float>(-hd * inv_w + dshift);
                    const float ys = yd * sc;
                    const __half a = __float2half_rn(ys);
                    mrow[i] = yd;
                    s0row[i] = a;
                    s1row[i] = __float2half_rn(ys - __half2float(a));
                    tr += static_cast<double>(yd);
                    sqd += static_cast<double>(yd) * yd;
                }
            }
            sq += static_cast<double>(sqr) + sqd;
        }
    };
    if (fp64) rows(std::integral_constant<int, 2>{});
    else if (fermi) rows(std::integral_constant<int, 1>{});
    else rows(std::integral_constant<int, 0>{});
    __shared__ double red[2][32];
    tr = warp_sum(tr);
    sq = warp_sum(sq);
    const int wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = tr; red[1][wid] = sq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
            a += red[0][w2];
            b += red[1][w2];
        }
        double *slot = pr.part + static_cast<size_t>(blockIdx.x) * kPartStride;
        slot[0] = a;
        slot[1] = b;
        slot[2] = 0.0;
        slot[3] = 0.0;
    }
}

// D = X (FP64) -> D_out, partials: slot[0] = tr D, slot[1] = sum Hp_ij D_ij.
__global__ void k_finalize(const MmaProb *probs, int prob, double *D, long long ldd) {
    const MmaProb &pr = probs[prob];
    const SolveState *st = pr.st;
    const int n = pr.n;
    const bool fermi = st->method == kMethodFermi;
    const bool from_x = st->x_fp64 != 0;
    const double *X = pr.Xd[st->xcur];
    const double c = st->c;
    // finite temperature: D = D0 + gamma Q (D0 = (I - z)/2 in Xd[0], Q = D0 - D0^2
    // in Xd[1]); gamma from the exact FP64 traces of the stored D0 and Q makes
    // tr D = N_e.  It is the first-order change of D for mu -> mu + gamma/beta.
    const double gamma = (fermi && st->tr_q > 0.0) ? (st->ne - st->tr_d0) / st->tr_q : 0.0;
    double tr = 0.0, eb = 0.0;
    // block b takes rows b, b + grid, ...; thread t the column pairs (2t, 2t + 1),
    // (2t + 2 blockDim, ...), ...: 16-byte accesses wherever a row is 16-byte
    // aligned (the D row for its store, the Hp row for its load)
    auto d_at = [&](int i, int j) -> double {
        if (fermi) {
            const long long at = static_cast<long long>(i) * pr.ldx + j;
            return pr.Xd[0][at] + gamma * pr.Xd[1][at];
        }
        if (from_x) return X[static_cast<long long>(i) * pr.ldx + j];
        return static_cast<double>(pr.Y[static_cast<long long>(i) * pr.ldy + j]) + (i == j ? c : 0.0);
    };
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const double *hrow = pr.H + static_cast<long long>(i) * pr.ldh;
        double *drow = D ? D + static_cast<long long>(i) * ldd : nullptr;
        const bool h16 = (reinterpret_cast<uintptr_t>(hrow) & 15u) == 0;
        const bool d16 = drow && (reinterpret_cast<uintptr_t>(drow) & 15u) == 0;
        for (int j = 2 * threadIdx.x; j < n; j += 2 * blockDim.x) {
            const bool two = j + 1 < n;
            const double d0 = d_at(i, j), d1 = two ? d_at(i, j + 1) : 0.0;
            double h0, h1 = 0.0;
            if (two && h16) {
                const double2 hv = *reinterpret_cast<const double2 *>(hrow + j);
                h0 = hv.x;
                h1 = hv.y;
            } else {
                h0 = hrow[j];
                if (two) h1 = hrow[j + 1];
            }
            if (drow) {
                if (two && d16) {
                    *reinterpret_cast<double2 *>(drow + j) = make_double2(d0, d1);
                } else {
                    drow[j] = d0;
                    if (two) drow[j + 1] = d1;
                }
            }
            if (i == j) tr += d0;
            if (i == j + 1) tr += d1;
            eb = fma(d0, h0, fma(d1, h1, eb));
        }
    }
    __shared__ double red[2][32];
    tr = warp_sum(tr);
    eb = warp_sum(eb);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][wid] = tr; red[1][wid] = eb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) { a += red[0][w2]; b += red[1][w2]; }
        double *slot = pr.part + static_cast<size_t>(blockIdx.x) * kPartStride;
        slot[0] = a;
        slot[1] = b;
    }
}

__global__ void k_finalize_reduce(const MmaProb *probs, int prob) {
    const MmaProb &pr = probs[prob];
    SolveState *st = pr.st;
    __shared__ double s_tr[512], s_eb[512];
    const int t = threadIdx.x;
    double tr = 0.0, eb = 0.0;
    for (int b = t; b < kFinBlocks; b += blockDim.x) {
        tr += pr.part[static_cast<size_t>(b) * kPartStride + 0];
        eb += pr.part[static_cast<size_t>(b) * kPartStride + 1];
    }
    s_tr[t] = tr;
    s_eb[t] = eb;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) { s_tr[t] += s_tr[t + o]; s_eb[t] += s_eb[t + o]; }
        __syncthreads();
    }
    if (t == 0) {
        st->trace = s_tr[0];
        st->e_band = s_eb[0];
        if (st->method == kMethodFermi && st->tr_q > 0.0)
            st->mu = st->mu_t + (st->ne - st->tr_d0) / st->tr_q / st->beta;
    }
}

__global__ void k_make_slices(const float *Y, int n, int ldy, float s, __half *hi, __half *lo,
                              int lds) {
    const long long total = static_cast<long long>(n) * n;
    for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / n);
        const int j = static_cast<int>(e - static_cast<long long>(i) * n);
        const float ys = Y[static_cast<long long>(i) * ldy + j] * s;
        const __half h = __float2half_rn(ys);
        hi[static_cast<long long>(i) * lds + j] = h;
        if (lo) lo[static_cast<long long>(i) * lds + j] = __float2half_rn(ys - __half2float(h));
    }
}

}  // namespace fe
