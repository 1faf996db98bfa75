// The products on either side of the density-matrix step in Chebyshev-
// filtered subspace iteration (Sec. I and Sec. III-A): the Rayleigh-Ritz
// projection Hp = Psi^T (H Psi) that forms the input of the expansion, and
// the rotation Psi D that uses its output (density or subspace update).
// Psi is the m x n block of filtered vectors (m grid points, m >> n).
//
// Both are contractions C = A B^T over a K dimension, A and B given as K-major
// FP16 slices (hi + lo of s X, 22-bit operands, s a power of two from max|X|),
// computed on the 5th-generation tensor cores with FP32 accumulation:
//   projection: A = Psi^T, B = (H Psi)^T (both n x m, K = m), C symmetric n x n
//               (upper tiles, mirrored); the long K is cut into nsplit parts
//               whose FP32 partial tiles are summed in FP64, in a fixed order,
//               by k_gemm_reduce (split-K: more work units to balance over the
//               SMs, and shorter FP32 sums);
//   rotation:   A = Psi (m x n, K = n), B = D (n x n, symmetric), C = Psi D
//               written in FP64 by the epilogue.
// As in the expansion's kernel, an accumulator in tensor memory lives for one
// 64-wide K chunk (cross terms hi*lo, lo*hi first, hi*hi last) and the chunks
// are summed in registers with round-to-nearest.
//
// Tiles are 128 rows (TMEM lanes) x 192 columns.  Warp roles (512 threads):
//   warp 0      TMA producer: per K chunk one box per slice for the A panel
//               (128 rows) and the B panel (192 rows), two stages of 80 KiB;
//   warp 1      TMEM owner and MMA issuer: per chunk 4 x 3 MMAs M128 N192 K16
//               into one of two 192-column chunk buffers;
//   warps 2-3   idle;
//   warps 4-15  drain + epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31
//               and columns 64 ((w - 4) / 4) .. +63 of the chunk.
// Every wait is bounded; on a timeout the kernel records an error code,
// waits (bounded) for its own copies and products in flight, frees TMEM and
// returns.
#include <cfloat>

#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {

namespace {

constexpr int kGA = kTileM * kTileK * 2;   // 16 KiB: one A slice of a stage
constexpr int kGB = kGemmN * kTileK * 2;   // 24 KiB: one B slice of a stage
constexpr int kGemmDrain0 = 4;             // first drain warp

struct alignas(1024) GemmStage {
    uint8_t a[kMaxSlices][kGA];
    uint8_t b[kMaxSlices][kGB];
};
static_assert(sizeof(GemmStage) % 1024 == 0 && kGA % 1024 == 0 && kGB % 1024 == 0,
              "128-byte swizzled tiles start on 1024-byte boundaries");

struct GemmTail {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t cfull[2];
    uint64_t cempty[2];
    uint32_t tmem_base;
    int pad;
    double stage[kGemmDrainWarps][32 * 9];  // per-warp staging of 32 rows x 8 columns
};

constexpr size_t kGemmSmemBytes = 1024 + sizeof(GemmStage) * kStages + sizeof(GemmTail);

__device__ __forceinline__ void record_error(DevCtl *ctl, int code) { atomicCAS(&ctl->err, 0, code); }

// power-of-two slice scale s with max|s X| < 2^14 (FP16 slices stay finite)
__device__ __forceinline__ double slice_scale_of(unsigned long long maxbits) {
    double m = __longlong_as_double(static_cast<long long>(maxbits));
    if (!(m > 0.0)) m = 1.0;
    int e;
    frexp(m, &e);  // m < 2^e
    return ldexp(1.0, 14 - e);
}

// The K-chunk range of work unit u: part u / ntiles of tile u % ntiles.
// The parts go outermost, so the work units that run at the same time
// (consecutive u over the CTAs) read the same K range of their panels: one
// part of every panel fits L2 and is read from DRAM about once per wave.
struct Unit {
    int tile, k0, k1;
};

__device__ __forceinline__ Unit unit_of(const GemmArgs &g, int u) {
    const int S = g.nsplit > 0 ? g.nsplit : 1;
    const int nk = (g.kdim + kTileK - 1) / kTileK;
    const int cs = (nk + S - 1) / S;
    Unit r;
    r.tile = u % g.ntiles;
    r.k0 = (u / g.ntiles) * cs;
    r.k1 = min(nk, r.k0 + cs);
    return r;
}

}  // namespace

__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_split(const GemmArgs *__restrict__ args, const TileEnt *__restrict__ tiles, DevCtl *ctl) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base_u32 = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
    GemmStage *stages = reinterpret_cast<GemmStage *>(smem);
    GemmTail *tail = reinterpret_cast<GemmTail *>(smem + sizeof(GemmStage) * kStages);
    const GemmArgs &g = *args;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t wait_ns = ctl->wait_ns;
    const int S = g.nsplit > 0 ? g.nsplit : 1;
    const int nunits = g.ntiles * S;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&tail->full[s], 1);
            mbar_init(&tail->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tail->cfull[a], 1);
            mbar_init(&tail->cempty[a], kGemmDrainWarps);
        }
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
        uint32_t last_phase[kStages];
        bool issued[kStages];
        for (int s = 0; s < kStages; ++s) { issued[s] = false; last_phase[s] = 0; }
        constexpr uint32_t bytes = static_cast<uint32_t>(kMaxSlices * (kGA + kGB));
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const Unit un = unit_of(g, u);
            const TileEnt te = tiles[un.tile];
            for (int kc = un.k0; kc < un.k1; ++kc) {
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
                    for (int s = 0; s < kMaxSlices; ++s) {
                        tma_load_2d(stages[stage].a[s], &g.tA[s], &tail->full[stage], kc * kTileK, te.I * kTileM);
                        tma_load_2d(stages[stage].b[s], &g.tB[s], &tail->full[stage], kc * kTileK, te.Jp * kGemmN);
                    }
                }
                __syncwarp();
                issued[stage] = true;
                last_phase[stage] = phase;
                if (++stage == kStages) { stage = 0; phase ^= 1u; }
            }
        }
        if (!ok && lane == 0) {
            // no TMA write may still be in flight when the CTA exits
            for (int s = 0; s < kStages; ++s)
                if (issued[s]) (void)mbar_wait_bounded(&tail->full[s], last_phase[s], wait_ns);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        uint32_t stage = 0, phase = 0, chunk = 0;
        bool ok = true, any_commit = false;
        constexpr uint32_t idesc = idesc_f16(kTileM, kGemmN, 0);
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const Unit un = unit_of(g, u);
            for (int kc = un.k0; kc < un.k1; ++kc) {
                const uint32_t buf = chunk & 1u;
                const uint32_t cph = (chunk >> 1) & 1u;
                bool got = true;
                if (lane == 0) got = mbar_wait_bounded(&tail->cempty[buf], cph ^ 1u, wait_ns);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (got) {
                    if (lane == 0) got = mbar_wait_bounded(&tail->full[stage], phase, wait_ns);
                    got = __shfl_sync(0xffffffffu, got, 0);
                    if (!got && lane == 0) record_error(ctl, kErrTimeoutFull);
                } else if (lane == 0) {
                    record_error(ctl, kErrTimeoutTmem);
                }
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t tmem_d = tmem_base + buf * kGemmN;
                    const uint64_t a0 = smem_desc_sw128(stages[stage].a[0]);
                    const uint64_t a1 = smem_desc_sw128(stages[stage].a[1]);
                    const uint64_t b0 = smem_desc_sw128(stages[stage].b[0]);
                    const uint64_t b1 = smem_desc_sw128(stages[stage].b[1]);
                    uint32_t accum = 0;
                    // small cross terms first: hi * lo, lo * hi
#pragma unroll
                    for (int kk = 0; kk < kTileK / 16; ++kk) {
                        const uint64_t off = static_cast<uint64_t>(kk * 2);  // 32 B along K
                        tc_mma_f16(tmem_d, a0 + off, b1 + off, idesc, accum);
                        accum = 1;
                        tc_mma_f16(tmem_d, a1 + off, b0 + off, idesc, accum);
                    }
                    // the full-magnitude hi * hi terms last
#pragma unroll
                    for (int kk = 0; kk < kTileK / 16; ++kk) {
                        const uint64_t off = static_cast<uint64_t>(kk * 2);
                        tc_mma_f16(tmem_d, a0 + off, b0 + off, idesc, 1u);
                    }
                    tc_commit(&tail->empty[stage]);  // smem stage may be refilled
                    tc_commit(&tail->cfull[buf]);    // chunk ready for the drain
                    any_commit = true;
                }
                __syncwarp();
                if (++stage == kStages) { stage = 0; phase ^= 1u; }
                ++chunk;
            }
        }
        if (!ok) {
            // every issued MMA must finish before TMEM is released
            if (lane == 0 && any_commit) {
                uint64_t *drain = &tail->cfull[chunk & 1u];
                tc_commit(drain);
                (void)mbar_wait_bounded(drain, (chunk >> 1) & 1u, wait_ns);
            }
            __syncwarp();
        }
    } else if (warp >= kGemmDrain0) {
        // ------------------------------------------------------------ drain + epilogue
        const int ew = warp - kGemmDrain0;   // 0..11
        const int q = warp & 3;              // TMEM lane quadrant (hardware rule: warp % 4)
        const int t3 = ew >> 2;              // column third of the tile: 64 columns
        uint32_t chunk = 0;
        bool ok = true;
        double inv = 1.0;
        if (g.nsplit == 0) inv = 1.0 / (slice_scale_of(g.amax[0]) * slice_scale_of(g.amax[1]));
        double *stg = tail->stage[ew];
        const int rsub = lane >> 3, csub = lane & 7;
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const Unit un = unit_of(g, u);
            const TileEnt te = tiles[un.tile];
            float acc[64];
#pragma unroll
            for (int c = 0; c < 64; ++c) acc[c] = 0.0f;
            for (int kc = un.k0; kc < un.k1; ++kc) {
                const uint32_t buf = chunk & 1u;
                const uint32_t cph = (chunk >> 1) & 1u;
                bool got = mbar_wait_bounded(&tail->cfull[buf], cph, wait_ns);
                got = __all_sync(0xffffffffu, got);
                if (!got) {
                    if (lane == 0) record_error(ctl, kErrTimeoutTmem);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + buf * kGemmN +
                                       static_cast<uint32_t>(t3 * 64);
#pragma unroll
                for (int c2 = 0; c2 < 2; ++c2) {
                    float v[32];
                    tmem_ld32(tbase + c2 * 32, v);
#pragma unroll
                    for (int x = 0; x < 32; ++x) acc[c2 * 32 + x] += v[x];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tail->cempty[buf]);
                ++chunk;
            }
            if (!ok) break;
            if (g.nsplit > 0) {
                // FP32 partial tile of this unit, [column][row]: a column's 32
                // rows of this warp are 128 consecutive bytes
                float *w = g.ws + static_cast<size_t>(u) * (kTileM * kGemmN) +
                           static_cast<size_t>(t3 * 64) * kTileM + q * 32 + lane;
#pragma unroll
                for (int c = 0; c < 64; ++c) w[static_cast<size_t>(c) * kTileM] = acc[c];
                continue;
            }
            // direct FP64 output C[i][j], i < rows_a, j < rows_b: each 8-column
            // group goes through the warp's staging buffer so that one store
            // instruction covers 4 rows x 8 consecutive columns
            const int i0 = te.I * kTileM + q * 32;
            const int cb = te.Jp * kGemmN + t3 * 64;
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) {
#pragma unroll
                for (int x = 0; x < 8; ++x) stg[lane * 9 + x] = static_cast<double>(acc[c8 * 8 + x]) * inv;
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int ii = i0 + 4 * k + rsub, jj = cb + c8 * 8 + csub;
                    if (ii < g.rows_a && jj < g.rows_b)
                        g.C[static_cast<long long>(ii) * g.ldc + jj] = stg[(4 * k + rsub) * 9 + csub];
                }
                __syncwarp();
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

// Sum of the nsplit FP32 partial tiles of every tile in a fixed order (FP64),
// scaled back by 1 / (s_A s_B), written to the upper part of the symmetric C
// and mirrored.  One block per tile.
__global__ void __launch_bounds__(256) k_gemm_reduce(const GemmArgs *__restrict__ args,
                                                     const TileEnt *__restrict__ tiles) {
    const GemmArgs &g = *args;
    const TileEnt te = tiles[blockIdx.x];
    const int S = g.nsplit;
    const double inv = 1.0 / (slice_scale_of(g.amax[0]) * slice_scale_of(g.amax[1]));
    const size_t tsz = static_cast<size_t>(kTileM) * kGemmN;
    const float *base = g.ws + static_cast<size_t>(blockIdx.x) * tsz;  // part s at unit s * ntiles + tile
    const size_t pstride = static_cast<size_t>(g.ntiles) * tsz;
    const int n = g.rows_a;
    for (int idx = threadIdx.x; idx < kTileM * kGemmN; idx += blockDim.x) {
        const int r = idx % kTileM, c = idx / kTileM;
        const int i = te.I * kTileM + r, j = te.Jp * kGemmN + c;
        if (i >= n || j >= n || j < i) continue;
        double sum = 0.0;
        for (int s = 0; s < S; ++s) sum += static_cast<double>(base[s * pstride + idx]);
        const double v = sum * inv;
        g.C[static_cast<long long>(i) * g.ldc + j] = v;
        if (j != i) g.C[static_cast<long long>(j) * g.ldc + i] = v;
    }
}

// max |X_ij| over a rows x cols block (ld) as the bit pattern of a
// non-negative FP64 value (ordered like the value), atomically into *out.
// Block b takes rows b, b + grid, ...; threads stride the columns, four
// loads in flight each.
__global__ void __launch_bounds__(256) k_absmax(const double *__restrict__ X, long long rows, long long cols,
                                                long long ld, unsigned long long *out) {
    constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long m = 0;
    const int t = threadIdx.x, nt = blockDim.x;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const double *row = X + r * ld;
        long long c = t;
        for (; c + 3 * nt < cols; c += 4 * nt) {
            const unsigned long long b0 = static_cast<unsigned long long>(__double_as_longlong(row[c])) & kAbs;
            const unsigned long long b1 = static_cast<unsigned long long>(__double_as_longlong(row[c + nt])) & kAbs;
            const unsigned long long b2 = static_cast<unsigned long long>(__double_as_longlong(row[c + 2 * nt])) & kAbs;
            const unsigned long long b3 = static_cast<unsigned long long>(__double_as_longlong(row[c + 3 * nt])) & kAbs;
            m = max(max(m, max(b0, b1)), max(b2, b3));
        }
        for (; c < cols; c += nt)
            m = max(m, static_cast<unsigned long long>(__double_as_longlong(row[c])) & kAbs);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

namespace {

// hi = fp16(s x), lo = fp16(s x - hi) with s x formed in FP32 (s a power of
// two): hi + lo equals x to 2^-24 relative besides the FP32 rounding of x
__device__ __forceinline__ void split_pair(double x0, double x1, float s, __half2 &h, __half2 &l) {
    const float y0 = f64_to_f32_rn(x0) * s, y1 = f64_to_f32_rn(x1) * s;
    h = __floats2half2_rn(y0, y1);
    const float2 back = __half22float2(h);
    l = __floats2half2_rn(y0 - back.x, y1 - back.y);
}

}  // namespace

// FP16 slices hi = fp16(s x), lo = fp16(s x - hi) of a rows x cols FP64 block,
// s from *amax.
// transpose = 0: out[r][c] (ld lds): block b takes rows b, b + grid, ...,
// each thread a pair of columns per pass (one 4-byte store per slice).
// transpose = 1: out[c][r]: 64 x 64 tiles through shared memory (stored by
// column, so that an output row of the tile is 64 consecutive values: 128
// bytes per slice and warp).  Blocks of 256 threads.
__global__ void __launch_bounds__(256) k_split_rows(const double *__restrict__ X, long long rows, long long cols,
                                                    long long ld, const unsigned long long *amax, __half *hi,
                                                    __half *lo, long long lds, int transpose) {
    __shared__ double t[64][65];
    const float s = static_cast<float>(slice_scale_of(*amax));
    const int tid = threadIdx.x;
    if (!transpose) {
        for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
            const double *row = X + r * ld;
            __half2 *h2 = reinterpret_cast<__half2 *>(hi + r * lds);
            __half2 *l2 = reinterpret_cast<__half2 *>(lo + r * lds);
            for (long long c = 2 * tid; c < cols; c += 2 * blockDim.x) {
                const double x0 = row[c], x1 = (c + 1 < cols) ? row[c + 1] : 0.0;
                __half2 h, l;
                split_pair(x0, x1, s, h, l);
                h2[c >> 1] = h;  // lds is even: the pair (c, c + 1) is one aligned 4-byte word
                l2[c >> 1] = l;
            }
        }
        return;
    }
    const int tx = tid & 31, ty = tid >> 5;  // 32 x 8
    const long long tiles_c = (cols + 63) / 64;
    const long long ntiles = ((rows + 63) / 64) * tiles_c;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long r0 = (tile / tiles_c) * 64, c0 = (tile % tiles_c) * 64;
        // load 64 rows x 64 columns (two columns per lane), keep them by column
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long r = r0 + ty + 8 * k;
            const long long c = c0 + 2 * tx;
            double x0 = 0.0, x1 = 0.0;
            if (r < rows) {
                if (c < cols) x0 = X[r * ld + c];
                if (c + 1 < cols) x1 = X[r * ld + c + 1];
            }
            t[2 * tx][ty + 8 * k] = x0;
            t[2 * tx + 1][ty + 8 * k] = x1;
        }
        __syncthreads();
        // output rows c0 .. c0 + 63, columns r0 .. r0 + 63: two columns per lane
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long c = c0 + ty + 8 * k;
            const long long r = r0 + 2 * tx;
            if (c < cols && r < rows) {
                __half2 h, l;
                split_pair(t[ty + 8 * k][2 * tx], t[ty + 8 * k][2 * tx + 1], s, h, l);
                reinterpret_cast<__half2 *>(hi + c * lds)[r >> 1] = h;  // lds even, r even
                reinterpret_cast<__half2 *>(lo + c * lds)[r >> 1] = l;
            }
        }
        __syncthreads();
    }
}

size_t gemm_smem_bytes() { return kGemmSmemBytes; }

}  // namespace fe
