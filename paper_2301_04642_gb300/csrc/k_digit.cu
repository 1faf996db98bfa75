// FP64-accurate SP2 step on the tensor cores (the polishing products of the
// mixed schedule; Sec. III-A runs the last iterations in FP64).
//
// GB300's FP64 units deliver about 1.25 TFLOP/s, so the FP64-accurate
// product X^2 is computed on the FP16 tensor cores instead, in exact integer
// arithmetic.  X/4 is written in fixed point with kDigits = 7 balanced
// base-256 digits,
//     X/4 = sum_{a=0}^{6} S_a 2^(-8(a+1)),   S_a integer in [-128, 127],
// each digit matrix held exactly in FP16.  Then
//     (X/4)^2 = sum_L 2^(-8(L+2)) sum_{a+c=L} S_a S_c^T
// and the levels L = 0..6 (28 digit products) are kept; the dropped levels
// are below 2^-64 relative to the leading one.  A digit product is an exact
// integer below 2^14, and a level sums at most 7 pairs, so over a K block of
// 128 its value stays below 7 * 128 * 2^14 < 2^24: the FP32 tensor-memory
// accumulator holds it exactly whatever its rounding.  Every K block each
// level buffer is drained into a per-element int64 fixed-point sum (unit
// 2^-64), and the epilogue forms P = X^2 = sum * 2^-60 in FP64.
//
// The epilogue is the SP2 update of the FP64-accurate step:
//     X' = (X^2 or 2X - X^2) + gamma (X - X^2)
// written to the other FP64 buffer (and mirrored), with per-tile partials
// tr X', ||X'||_F^2 and ||X^2 - X||_F^2 (same slots as the SIMT FP64 step).
// As the first product of a polishing pair it also writes the FP16 slices of
// Delta = X^2 - X and of S (the operands of the pair's second, split-FP16
// product; see the control kernel).
//
// Tiles: 128 rows (block I) x 64 columns (block J), J >= 2I, one persistent
// CTA per SM.  Warp roles as in the split-FP16 kernel: warp 0 TMA (per K
// stage of kDigitK one box per digit for A and for B; kDigitStages stages),
// warp 1 TMEM owner and MMA
// issuer (7 level buffers of 64 columns), warps 2-9 drain + epilogue (warp w:
// TMEM lanes 32 (w % 4) .., columns 32 ((w - 2) / 4) .. of each level).
// Every wait is bounded; on a timeout the kernel records an error code,
// drains its own copies and MMAs, frees TMEM and returns.
#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {

namespace {

constexpr int kDA = kTileM * kDigitK * 2;   // one digit, 128 rows x kDigitK
constexpr int kDB = kDigitN * kDigitK * 2;  // one digit, 64 rows x kDigitK
static_assert(kDigitK == 16 || kDigitK == 32, "a stage is one 32- or 64-byte swizzle row");

// shared-memory descriptor of one digit block of a stage (K-major, swizzled
// rows of kDigitK FP16)
__device__ __forceinline__ uint64_t digit_desc(const void *tile) {
    if constexpr (kDigitK == 16) return smem_desc_sw32(tile);
    else return smem_desc_sw64(tile);
}
constexpr int kStagesPerBlock = kDigitKBlock / kDigitK;

struct alignas(1024) DigitStage {
    uint8_t a[kDigits][kDA];
    uint8_t b[kDigits][kDB];
};

struct DigitTail {
    uint64_t full[kDigitStages];
    uint64_t empty[kDigitStages];
    uint64_t lfull[kDigits];
    uint64_t lfree[kDigits];
    uint64_t abort_bar;
    uint32_t tmem_base;
    int abort_flag;
    double red[kEpiWarps][4];
    int vote[kEpiWarps];
    double stage[kEpiWarps][32 * 9];
};

constexpr size_t kDigitSmemBytes = 1024 + sizeof(DigitStage) * kDigitStages + sizeof(DigitTail);

__device__ __forceinline__ int step_kind(const SolveState *st) {
    return *reinterpret_cast<const volatile int *>(&st->kind);
}

__device__ __forceinline__ void record_error(DevCtl *ctl, int code) { atomicCAS(&ctl->err, 0, code); }

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// The current iterate at (i, j): Xd[xcur] once FP64, else c I + Y.
__device__ __forceinline__ double x_at(const MmaProb &pr, const SolveState *st, int i, int j) {
    if (st->x_fp64) return pr.Xd[st->xcur][static_cast<size_t>(i) * pr.ldx + j];
    return static_cast<double>(pr.Y[static_cast<size_t>(i) * pr.ldy + j]) + (i == j ? st->c : 0.0);
}

// round(x 2^54) by integer operations on the FP64 encoding (GB300's FP64
// conversions are slow), clamped to |x| <= 1.98 so that the top digit of the
// balanced base-256 expansion stays in [-128, 127]
__device__ __forceinline__ long long fixed54(double x) {
    constexpr long long kLim = 35668509048774328LL;  // 1.98 * 2^54
    const long long bits = __double_as_longlong(x);
    const int e = static_cast<int>((bits >> 52) & 0x7FF);
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);  // |x| = m 2^(e - 1075)
    const int sh = e - 1021;                                       // |x| 2^54 = m 2^sh
    long long v;
    if (e == 0) v = 0;                  // zero or subnormal
    else if (sh > 2) v = kLim;          // |x| >= 4, Inf, NaN
    else if (sh >= 0) v = m << sh;
    else if (sh > -63) v = (m + (1LL << (-sh - 1))) >> (-sh);  // round half away from zero
    else v = 0;
    v = v > kLim ? kLim : v;
    return bits < 0 ? -v : v;
}

}  // namespace

// round(y 2^54) for an FP32 y, by integer operations on its encoding: the
// same value fixed54 gives for the (exact) FP64 widening of y
__device__ __forceinline__ long long fixed54_f(float y) {
    constexpr long long kLim = 35668509048774328LL;  // 1.98 * 2^54
    const unsigned bits = __float_as_uint(y);
    const int e = static_cast<int>((bits >> 23) & 0xFFu);
    const long long m = static_cast<long long>((bits & 0x7FFFFFu) | 0x800000u);  // |y| = m 2^(e - 150)
    const int sh = e - 96;                                                        // |y| 2^54 = m 2^sh
    long long v;
    if (e == 0) v = 0;                  // zero or subnormal (below 2^-126)
    else if (sh > 31) v = kLim;         // |y| >= 2^9, Inf, NaN
    else if (sh >= 0) v = m << sh;
    else if (sh > -25) v = (m + (1LL << (-sh - 1))) >> (-sh);  // round half away from zero
    else v = 0;
    v = v > kLim ? kLim : v;
    return (bits >> 31) ? -v : v;
}

// balanced base-256 digits of V (least significant first), two elements at a time
__device__ __forceinline__ void put_digits2(const MmaProb &pr, size_t at, long long V0, long long V1) {
#pragma unroll
    for (int a = kDigits - 1; a >= 0; --a) {
        const long long d0 = ((V0 + 128) & 255) - 128, d1 = ((V1 + 128) & 255) - 128;
        *reinterpret_cast<__half2 *>(pr.dig[a] + at) =
            __halves2half2(__int2half_rn(static_cast<int>(d0)), __int2half_rn(static_cast<int>(d1)));
        V0 = (V0 - d0) >> 8;
        V1 = (V1 - d1) >> 8;
    }
}

__global__ void k_digit_prep(const MmaProb *probs, int nprobs) {
    for (int p = 0; p < nprobs; ++p) {
        const MmaProb &pr = probs[p];
        const SolveState *st = pr.st;
        if (step_kind(st) != kDigit) continue;
        const int n = pr.n;
        const bool xf = st->x_fp64 != 0;
        // V = round(X/4 * 2^56) = round(x 2^54), two adjacent columns per
        // thread (lds is even: one 4-byte store per digit array); off the
        // diagonal the FP32 iterate c I + Y is just Y, converted without FP64
        // arithmetic, and the diagonal takes the FP64 sum y + c
        // four column pairs per thread are loaded before any is converted
        // (enough bytes in flight for the HBM rate with 2 blocks per SM)
        const int cs = 2 * blockDim.x;
        const double c = st->c;
        for (int i = blockIdx.x; i < n; i += gridDim.x) {
            const double *X = pr.Xd[st->xcur] + static_cast<size_t>(i) * pr.ldx;
            const float *Yr = pr.Y + static_cast<size_t>(i) * pr.ldy;
            for (int jb = 2 * threadIdx.x; jb < n; jb += 4 * cs) {
                double a[4], b[4];  // FP64 iterate
                float fa[4], fb[4];  // or the FP32 small part (no FP64 conversion off the diagonal)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = jb + q * cs;
                    a[q] = 0.0;
                    b[q] = 0.0;
                    fa[q] = 0.0f;
                    fb[q] = 0.0f;
                    if (j < n) {
                        if (xf) {
                            a[q] = X[j];
                            if (j + 1 < n) b[q] = X[j + 1];
                        } else {
                            const float2 y2 = *reinterpret_cast<const float2 *>(Yr + j);  // ldy even
                            fa[q] = y2.x;
                            fb[q] = y2.y;
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = jb + q * cs;
                    if (j >= n) continue;
                    const bool two = j + 1 < n;
                    long long V0, V1 = 0;
                    if (xf) {
                        V0 = fixed54(a[q]);
                        if (two) V1 = fixed54(b[q]);
                    } else {
                        // off the diagonal the FP32 iterate c I + Y is just Y
                        V0 = (i == j) ? fixed54(static_cast<double>(fa[q]) + c) : fixed54_f(fa[q]);
                        if (two) V1 = (i == j + 1) ? fixed54(static_cast<double>(fb[q]) + c) : fixed54_f(fb[q]);
                    }
                    put_digits2(pr, static_cast<size_t>(i) * pr.lds + j, V0, V1);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kMmaThreads, 1)
    k_digit_mma(const MmaProb *__restrict__ probs, const TileEnt *__restrict__ tiles, int ntiles,
                DevCtl *ctl) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base_u32 = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
    DigitStage *stages = reinterpret_cast<DigitStage *>(smem);
    DigitTail *tail = reinterpret_cast<DigitTail *>(smem + sizeof(DigitStage) * kDigitStages);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t wait_ns = ctl->wait_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kDigitStages; ++s) {
            mbar_init(&tail->full[s], 1);
            mbar_init(&tail->empty[s], 1);
        }
        for (int l = 0; l < kDigits; ++l) {
            mbar_init(&tail->lfull[l], 1);
            mbar_init(&tail->lfree[l], kEpiWarps);
        }
        mbar_init(&tail->abort_bar, 1);
        tail->abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(&tail->tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tail->tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        uint32_t stage = 0, phase = 0;
        bool ok = true;
        uint32_t last_phase[kDigitStages];
        bool issued[kDigitStages];
        for (int s = 0; s < kDigitStages; ++s) { issued[s] = false; last_phase[s] = 0; }
        constexpr uint32_t bytes = static_cast<uint32_t>(kDigits * (kDA + kDB));
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TileEnt te = tiles[t];
            const MmaProb &pr = probs[te.prob];
            if (step_kind(pr.st) != kDigit) continue;
            const int nk = (pr.n + kDigitK - 1) / kDigitK;
            for (int kc = 0; kc < nk; ++kc) {
                bool got = true;
                if (lane == 0) got = mbar_wait_bounded(&tail->empty[stage], phase ^ 1u, wait_ns);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    if (lane == 0) record_error(ctl, kErrTimeoutEmpty);
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    mbar_expect_tx(&tail->full[stage], bytes);
                    for (int a = 0; a < kDigits; ++a) {
                        tma_load_2d(stages[stage].a[a], &pr.dA[a], &tail->full[stage], kc * kDigitK,
                                    te.I * kTileM);
                        tma_load_2d(stages[stage].b[a], &pr.dB[a], &tail->full[stage], kc * kDigitK,
                                    te.Jp * kDigitN);
                    }
                }
                __syncwarp();
                issued[stage] = true;
                last_phase[stage] = phase;
                if (++stage == kDigitStages) { stage = 0; phase ^= 1u; }
            }
        }
        if (!ok) {
            tail->abort_flag = 1;
            if (lane == 0)
                for (int s = 0; s < kDigitStages; ++s)
                    if (issued[s]) (void)mbar_wait_bounded(&tail->full[s], last_phase[s], wait_ns);
            __syncwarp();
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        uint32_t stage = 0, phase = 0;
        uint32_t blk = 0;  // K blocks of this CTA: level-buffer phase = blk & 1
        bool ok = true;
        bool any_commit = false;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TileEnt te = tiles[t];
            const MmaProb &pr = probs[te.prob];
            if (step_kind(pr.st) != kDigit) continue;
            const int nk = (pr.n + kDigitK - 1) / kDigitK;
            for (int kc = 0; kc < nk; ++kc) {
                const int sb = kc % kStagesPerBlock;
                const bool first = (sb == 0);
                const bool last = (sb == kStagesPerBlock - 1) || (kc == nk - 1);
                bool got = true;
                if (lane == 0) got = mbar_wait_bounded(&tail->full[stage], phase, wait_ns);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    if (lane == 0) record_error(ctl, kErrTimeoutFull);
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    uint64_t da[kDigits], db[kDigits];
#pragma unroll
                    for (int a = 0; a < kDigits; ++a) {
                        da[a] = digit_desc(stages[stage].a[a]);
                        db[a] = digit_desc(stages[stage].b[a]);
                    }
#pragma unroll
                    // A digit a against up to four B digits c0 .. c0 + w - 1 in
                    // one MMA of N = 64 w: those B tiles are adjacent in shared
                    // memory and levels a + c0 .. a + c0 + w - 1 are adjacent
                    // 64-column buffers.  Digit a = 0 meets every level first,
                    // so its MMAs start the block's sums (accumulate off at
                    // the first K step).
#pragma unroll
                    for (int a = 0; a < kDigits; ++a) {
#pragma unroll
                        for (int c0 = 0; c0 + a < kDigits; c0 += 4) {
                            const int L = a + c0;
                            const int w = (kDigits - L < 4) ? (kDigits - L) : 4;  // levels in this MMA
                            if (first && a == 0 && got) {
                                // the drain of these levels' previous block must be done
                                for (int l = L; l < L + w && got; ++l)
                                    got = mbar_wait_bounded(&tail->lfree[l], (blk & 1u) ^ 1u, wait_ns);
                                if (!got) record_error(ctl, kErrTimeoutTmem);
                            }
                            if (got) {
                                const uint32_t tmem_d = tmem_base + static_cast<uint32_t>(L * kDigitN);
                                const uint32_t id = idesc_f16(kTileM, w * kDigitN, 0);
#pragma unroll
                                for (int kk = 0; kk < kDigitK / 16; ++kk) {
                                    const uint64_t off = static_cast<uint64_t>(kk * 2);  // 32 B along K
                                    const uint32_t acc = (first && a == 0 && kk == 0) ? 0u : 1u;
                                    tc_mma_f16(tmem_d, da[a] + off, db[c0] + off, id, acc);
                                }
                                any_commit = true;
                            }
                        }
                        // digit a is the last to add to level a (c = 0)
                        if (last && got) tc_commit(&tail->lfull[a]);
                    }
                    tc_commit(&tail->empty[stage]);
                }
                got = __shfl_sync(0xffffffffu, got, 0);
                __syncwarp();
                if (!got) {
                    ok = false;
                    break;
                }
                if (++stage == kDigitStages) { stage = 0; phase ^= 1u; }
                if (last) ++blk;
            }
        }
        if (!ok) {
            tail->abort_flag = 1;
            // every issued MMA must finish before TMEM is released
            if (lane == 0 && any_commit) {
                tc_commit(&tail->abort_bar);
                (void)mbar_wait_bounded(&tail->abort_bar, 0, wait_ns);
            }
            __syncwarp();
        }
    } else {
        // ------------------------------------------------------------ drain + epilogue
        const int ew = warp - 2;
        const int q = warp & 3;                // TMEM lane quadrant (warp % 4)
        const int h = ew >> 2;                 // column half: 32 of the tile's 64
        uint32_t blk = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TileEnt te = tiles[t];
            const MmaProb &pr = probs[te.prob];
            const SolveState *st = pr.st;
            if (step_kind(st) != kDigit) continue;
            const int n = pr.n;
            const int nk = (n + kDigitK - 1) / kDigitK;
            const int nb = (nk + kStagesPerBlock - 1) / kStagesPerBlock;
            long long acc[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) acc[u] = 0;
            for (int b = 0; b < nb && ok; ++b) {
#pragma unroll 1
                for (int L = 0; L < kDigits; ++L) {
                    bool got = mbar_wait_bounded(&tail->lfull[L], blk & 1u, wait_ns);
                    got = __all_sync(0xffffffffu, got);
                    if (!got) {
                        if (lane == 0) record_error(ctl, kErrTimeoutTmem);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    float v[32];
                    tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                                  static_cast<uint32_t>(L * kDigitN + h * 32),
                              v);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tail->lfree[L]);
                    // level L carries unit 2^(-8(L+2)); the sum's unit is 2^-64
                    const int shift = 8 * (kDigits - 1 - L);
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const long long iv = static_cast<long long>(__float2int_rn(v[u]));
                        acc[u] += static_cast<long long>(static_cast<unsigned long long>(iv) << shift);
                    }
                }
                ++blk;
            }
            if (lane == 0) tail->vote[ew] = ok ? 1 : 0;
            epi_bar();
            bool all_ok = true;
            for (int w = 0; w < kEpiWarps; ++w) all_ok = all_ok && (tail->vote[w] != 0);
            epi_bar();
            if (!all_ok) {
                ok = false;
                break;
            }

            // ---- epilogue: X' = (X^2 or 2X - X^2) + gamma (X - X^2); the first
            // product of a polishing pair also writes the FP16 slices of
            // Delta0 = X^2 - X (slot Y0) and S = 2X + Delta0 (X^2 branch) or
            // 2I - 2X + Delta0 (slot Y1), the operands of the pair's second product
            const int sq = st->sq;
            const double gamma = st->gamma;
            double *Xo = pr.Xd[st->xcur ^ 1];  // the control kernel flips xcur afterwards
            const int ldx = pr.ldx, lds = pr.lds;
            const bool emit = st->pol_emit != 0;
            const float sD = st->pol_sD, sS = st->pol_sS;
            const MatSlot &mD = pr.mats[kMatY0];
            const MatSlot &mS = pr.mats[kMatY1];
            const int i0 = te.I * kTileM + q * 32;
            const int i = i0 + lane;
            const int j0 = te.Jp * kDigitN + h * 32;
            const int rsub = lane >> 3, csub = lane & 7;
            double tr = 0.0, s2 = 0.0, id = 0.0;
            double *stg = tail->stage[ew];
            // the (i, j) half goes through the staging buffer: 4 rows x 8
            // consecutive columns per store instruction
            auto put_staged = [&](int jg, int what) {
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int ii = i0 + 4 * k + rsub, jj = jg + csub;
                    if (ii < n && jj < n && jj >= ii) {
                        const double v = stg[(4 * k + rsub) * 9 + csub];
                        if (what == 0) {
                            Xo[static_cast<size_t>(ii) * ldx + jj] = v;
                        } else {
                            const MatSlot &m = (what == 1) ? mD : mS;
                            const float y = static_cast<float>(v) * ((what == 1) ? sD : sS);
                            const __half hh = __float2half_rn(y);
                            const size_t at = static_cast<size_t>(ii) * lds + jj;
                            m.sl[0][at] = hh;
                            m.sl[1][at] = __float2half_rn(y - __half2float(hh));
                        }
                    }
                }
                __syncwarp();
            };
            if (i0 < n && j0 < n && j0 + 31 >= i0) {
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const int jg = j0 + 8 * g;
                    double dv[8], sv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = jg + u;
                        double xn = 0.0;
                        dv[u] = 0.0;
                        sv[u] = 0.0;
                        if (i < n && j < n && j >= i) {
                            const double P = static_cast<double>(acc[8 * g + u]) * 8.673617379884035e-19;  // 2^-60
                            const double xo = x_at(pr, st, j, i);  // symmetric: coalesced read
                            xn = (sq ? P : 2.0 * xo - P) + gamma * (xo - P);
                            const double dd = P - xo;
                            dv[u] = dd;
                            sv[u] = (sq ? 2.0 * xo : ((j == i) ? 2.0 : 0.0) - 2.0 * xo) + dd;
                            if (j != i) {
                                Xo[static_cast<size_t>(j) * ldx + i] = xn;
                                s2 += 2.0 * xn * xn;
                                id += 2.0 * dd * dd;
                                if (emit) {
                                    const size_t at = static_cast<size_t>(j) * lds + i;
                                    const float yd = static_cast<float>(dd) * sD;
                                    const float ys = static_cast<float>(sv[u]) * sS;
                                    const __half hd = __float2half_rn(yd), hs = __float2half_rn(ys);
                                    mD.sl[0][at] = hd;
                                    mD.sl[1][at] = __float2half_rn(yd - __half2float(hd));
                                    mS.sl[0][at] = hs;
                                    mS.sl[1][at] = __float2half_rn(ys - __half2float(hs));
                                }
                            } else {
                                tr += xn;
                                s2 += xn * xn;
                                id += dd * dd;
                            }
                        }
                        stg[lane * 9 + u] = xn;
                    }
                    put_staged(jg, 0);
                    if (emit) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) stg[lane * 9 + u] = dv[u];
                        put_staged(jg, 1);
#pragma unroll
                        for (int u = 0; u < 8; ++u) stg[lane * 9 + u] = sv[u];
                        put_staged(jg, 2);
                    }
                }
            }
            tr = warp_sum(tr);
            s2 = warp_sum(s2);
            id = warp_sum(id);
            if (lane == 0) {
                tail->red[ew][0] = tr;
                tail->red[ew][1] = s2;
                tail->red[ew][2] = id;
            }
            epi_bar();
            if (ew == 0 && lane == 0) {
                double a = 0, b2 = 0, c = 0;
                for (int w = 0; w < kEpiWarps; ++w) {
                    a += tail->red[w][0];
                    b2 += tail->red[w][1];
                    c += tail->red[w][2];
                }
                double *slot = pr.part + static_cast<size_t>(te.slot) * kPartStride;
                slot[0] = a;
                slot[1] = b2;
                slot[2] = 0.0;
                slot[3] = c;
            }
            epi_bar();
        }
        if (!ok) tail->abort_flag = 1;
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

size_t digit_smem_bytes() { return kDigitSmemBytes; }

}  // namespace fe
