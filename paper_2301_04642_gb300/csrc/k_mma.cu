// Symmetric products on the 5th-generation tensor cores with the update of
// the expansion fused into the epilogue (Sec. II-B1 Eq. (1), Sec. II-B3;
// Sec. III-B: the matrix product dominates the cost).
//
// Every step multiplies two symmetric, mutually commuting matrices given by
// their small parts A~, B~ (the identity parts are FP64 scalars in the solve
// state), so the product is symmetric and only upper-triangle 128x128 blocks
// are computed.  (A~ B~)_ij = sum_k A~_ik B~_jk: both operands are row panels
// of K-major FP16 slice arrays, loaded by TMA with 128-byte swizzling.  The
// epilogue evaluates up to three outputs  a v + b1 E1 + b2 E2 + c [i == j]
// (v the product, E1/E2 FP32 masters), writes them as FP32 masters, FP16
// slices for the next step and/or FP64 matrices, mirrors every value to the
// lower triangle, and leaves per-tile FP64 partials (trace and squared
// Frobenius norm of one output, trace of another, and an auxiliary sum of
// squares used as the idempotency measure ||X^2 - X||_F^2).  The step to run
// is described by the ProdOp the control kernel wrote into the solve state.
//
// One persistent CTA per SM walks a list of tiles (of one or many problems).
// A problem's tile width bn is 256 (128 rows of block I x the blocks 2Jp,
// 2Jp+1) or 128 (block I x block J = Jp, J >= I), as the host's tile-shape
// table chose for its n; one launch may mix both.
//
// Accuracy: the tensor core adds every MMA into its FP32 accumulator with a
// one-sided rounding, so an accumulator that lives for the whole K loop
// collects an error that grows with K.  Here an accumulator lives for one
// 64-wide K chunk only: per chunk the small cross terms hi*lo and lo*hi are
// issued first and the four hi*hi MMAs last, so the truncating additions at
// full magnitude are four per chunk.  The drain warps read each chunk from
// TMEM and sum the chunks in registers (round-to-nearest FP32) while the MMA
// warp fills the other chunk buffer.
//
// Warp roles (384 threads; warpgroup 0 hands registers to warpgroups 1-2):
//   warp 0      TMA producer: per K chunk one box per slice for the A panel
//               (128 rows) and the B panel (bn rows).
//   warp 1      TMEM owner and MMA issuer: per chunk 4 x (1 or 3) MMAs
//               M128 Nbn K16 into one of two chunk buffers (2 x 256 cols).
//   warps 2-3   idle (give their registers away)
//   warps 4-11  drain + epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31
//               and the columns bn/2 ((w - 4) / 4) .. +bn/2-1 (one 128x128
//               block, or half of one when bn = 128) in 64-column loads.
// Every wait is bounded; on a timeout the kernel records an error code,
// drains its own copies and MMAs, frees TMEM and returns.
#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {

namespace {

struct alignas(1024) StageSmem {
    uint8_t a[kMaxSlices][kSliceABytes];
    uint8_t b[kMaxSlices][kSliceBBytes];
};

// The launch's schedule table, in shared memory when the launch has 2 to
// kSchedProbs problems: per problem (table order) the inclusive prefix sums
// of active tiles and of work units, and the units of one of its tiles (0:
// no tensor-core work in this step).  Built once per launch; without it every
// tile hand-out would walk the problem table in global memory, a chain of
// dependent loads per problem.
constexpr int kSchedProbs = 256;
struct SchedTab {
    long long units[kSchedProbs];
    int tiles[kSchedProbs];
    int w[kSchedProbs];
    int bnmin, wmin, wmax, pad;
};

// The fields of one output that the store loop's vector path reads.
struct OutCache {
    float a, b1, b2, s, g1r, g1c, g2r, g2c;
    int flags, pad;
    float *master;
    __half *sl0, *sl1;
};

struct MmaSmemTail {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t cfull[2];
    uint64_t cempty[2];
    uint32_t tmem_base;
    int abort_flag;
    double red[kEpiWarps][4];
    int vote[kEpiWarps];
    int sk_ticket, sk_ok;             // split-tile hand-off (drain warp 0 writes, all read)
    double stage[kEpiWarps][32 * 9];  // per-warp staging of 32 rows x 8 columns (direct writes)
    OutCache oc[kEpiWarps][3];        // per-warp copy of the step's outputs (shared-memory loads
                                      // in the store loop instead of reloads after every store)
    SchedTab sch;
};

constexpr size_t kMmaSmemBytes = 1024 + sizeof(StageSmem) * kStages + sizeof(MmaSmemTail);

__device__ __forceinline__ int step_kind(const SolveState *st) {
    return *reinterpret_cast<const volatile int *>(&st->kind);
}

__device__ __forceinline__ bool tile_active(const SolveState *st) {
    const int kind = step_kind(st);
    return kind == kTcSingle || kind == kTcSplit || kind == kTcElem || kind == kTcDelta;
}

// FP16 slices per operand: two for the split products
__device__ __forceinline__ int step_slices(const SolveState *st) {
    const int kind = step_kind(st);
    return (kind == kTcSplit || kind == kTcDelta) ? 2 : 1;
}

// K chunks of this step (0 for an epilogue-only step)
__device__ __forceinline__ int step_chunks(const SolveState *st, int n) {
    return step_kind(st) == kTcElem ? 0 : (n + kTileK - 1) / kTileK;
}

// tile width of a problem: 128 or 256 columns
__device__ __forceinline__ int tile_bn(const MmaProb &pr) { return pr.bn == kTileM ? kTileM : kTileN; }

__device__ __forceinline__ void record_error(DevCtl *ctl, int code) { atomicCAS(&ctl->err, 0, code); }

// named barrier of the 8 drain/epilogue warps
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// hi/lo FP16 slices of s * v[0..7], packed for one 16-byte store each
// (the same roundings as put_slices)
__device__ __forceinline__ void split8(const float *v, float s, uint4 &hv, uint4 &lv) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float y0 = v[2 * p] * s, y1 = v[2 * p + 1] * s;
        const __half2 hh = __floats2half2_rn(y0, y1);
        const float2 back = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(y0 - back.x, y1 - back.y);
        h[p] = *reinterpret_cast<const uint32_t *>(&hh);
        l[p] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    hv = make_uint4(h[0], h[1], h[2], h[3]);
    lv = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void put_slices(const MatSlot &m, size_t at, float ys) {
    const __half hh = __float2half_rn(ys);
    m.sl[0][at] = hh;
    m.sl[1][at] = __float2half_rn(ys - __half2float(hh));
}

// ---- Schedule: data-parallel waves, then Stream-K.  The launch's work is the
// sequence, over the active problems in table order, of their tiles, each
// worth `units` = its 64-wide K chunks (1 for an epilogue-only step) times its
// width over the narrowest width in the launch (so a 128 x 256 tile weighs
// twice a 128 x 128 one when both are present).
// When every tile is worth the same and there are at least two waves, whole
// waves go first, tile t to CTA t mod grid: all CTAs then step through K
// together on tiles that are neighbours in the list (the host orders tiles in
// bands so that these share row and column panels), and each panel chunk is
// read from HBM about once per wave while the rest hit L2.  The remaining one
// to two waves of tiles (all of them otherwise) are cut into equal contiguous
// ranges, one per participating CTA (Stream-K), so tile boundaries (and store
// phases) fall at different times in different CTAs and the last wave is not
// left half empty.  At most G = W / (largest tile) CTAs take part, so a tile
// spans at most two ranges: a head segment at the end of one CTA's range and
// a tail segment at the start of the next one's.  A chunk worth f units
// belongs to the range that holds its first unit; a range part that holds no
// chunk's first unit is skipped.  Every role of a CTA walks the same segments.
struct Seg {
    int tile;   // index into the launch's tile list
    int prob;   // index of its problem in the launch's table
    int k0;     // first chunk
    int nch;    // chunks (0 for an epilogue-only step)
    bool split; // the tile is shared with a neighbouring CTA
    bool head;  // this CTA has its first chunks (else its last)
};

// chunks of a tile, counting an epilogue-only step's tile as one
__device__ __forceinline__ int tile_chunks(const MmaProb &pr) {
    const int nk = step_chunks(pr.st, pr.n);
    return nk > 0 ? nk : 1;
}

// Fill the schedule table (every thread of the CTA calls this between two
// CTA barriers, `warp0` says whether it is in warp 0).  Pass 1, all threads:
// chunks, width and tiles of each problem.  Pass 2, warp 0 after a barrier:
// the narrowest width, the units per tile, and prefix sums (each lane scans
// a contiguous run of problems, then the run totals are scanned across the
// warp).
__device__ void sched_pass1(SchedTab *t, const MmaProb *probs, int np) {
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
        const MmaProb &pr = probs[q];
        const bool act = pr.tc_ntiles > 0 && tile_active(pr.st);
        t->w[q] = act ? tile_chunks(pr) : 0;
        t->tiles[q] = act ? pr.tc_ntiles : 0;
        t->units[q] = act ? tile_bn(pr) : 0;
    }
}

__device__ void sched_pass2(SchedTab *t, int np, int lane) {
    int bm = kTileN;
    for (int q = lane; q < np; q += 32)
        if (t->w[q] > 0) bm = static_cast<int>(t->units[q]) < bm ? static_cast<int>(t->units[q]) : bm;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int y = __shfl_xor_sync(0xffffffffu, bm, o);
        bm = y < bm ? y : bm;
    }
    const int per = (np + 31) / 32;
    const int q0 = lane * per, q1 = (q0 + per < np) ? q0 + per : np;
    long long su = 0;
    int st = 0, wmin = 0x7fffffff, wmax = 1;
    for (int q = q0; q < q1; ++q) {
        const int c = t->w[q];
        const int w = c > 0 ? c * (static_cast<int>(t->units[q]) / bm) : 0;
        if (c > 0) {
            wmin = w < wmin ? w : wmin;
            wmax = w > wmax ? w : wmax;
        }
        su += static_cast<long long>(t->tiles[q]) * w;
        st += t->tiles[q];
        t->w[q] = w;
        t->units[q] = su;
        t->tiles[q] = st;
    }
    long long eu = su;
    int et = st;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long yu = __shfl_up_sync(0xffffffffu, eu, o);
        const int yt = __shfl_up_sync(0xffffffffu, et, o);
        if (lane >= o) {
            eu += yu;
            et += yt;
        }
    }
    eu -= su;
    et -= st;
    for (int q = q0; q < q1; ++q) {
        t->units[q] += eu;
        t->tiles[q] += et;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int a = __shfl_xor_sync(0xffffffffu, wmin, o);
        const int b = __shfl_xor_sync(0xffffffffu, wmax, o);
        wmin = a < wmin ? a : wmin;
        wmax = b > wmax ? b : wmax;
    }
    if (lane == 0) {
        t->bnmin = bm;
        t->wmin = wmin;
        t->wmax = wmax;
    }
}

struct SegIter {
    const MmaProb *probs;
    const SchedTab *tab;   // the shared-memory table, or null: walk the table in global memory
    int nprobs;
    int bnmin;             // narrowest tile width among the active problems
    long long dp, dp_end;  // data-parallel part: next tile index (over active tiles), end
    long long g, end;      // Stream-K part: this CTA's range of work units

    __device__ int unit_f(const MmaProb &pr) const { return tile_bn(pr) / bnmin; }
    __device__ int tile_units(const MmaProb &pr) const { return tile_chunks(pr) * unit_f(pr); }

    // the problem holding active tile r (tiles = true) or work unit r of the
    // launch, with r made relative to the problem's first; nprobs if none
    __device__ int find(long long &r, bool tiles) const {
        if (nprobs <= 0) return nprobs;
        if (tab) {
            int lo = 0, hi = nprobs - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const long long v = tiles ? tab->tiles[mid] : tab->units[mid];
                if (v > r) hi = mid;
                else lo = mid + 1;
            }
            const long long v = tiles ? tab->tiles[lo] : tab->units[lo];
            if (v <= r) return nprobs;
            if (lo > 0) r -= tiles ? tab->tiles[lo - 1] : tab->units[lo - 1];
            return lo;
        }
        for (int q = 0; q < nprobs; ++q) {
            const MmaProb &pr = probs[q];
            if (pr.tc_ntiles == 0 || !tile_active(pr.st)) continue;
            const long long span = tiles ? pr.tc_ntiles : static_cast<long long>(pr.tc_ntiles) * tile_units(pr);
            if (r < span) return q;
            r -= span;
        }
        return nprobs;
    }

    __device__ void init(const MmaProb *p, int np, const SchedTab *t) {
        probs = p;
        nprobs = np;
        tab = t;
        long long W = 0, T = 0;
        int wmax = 1, wmin = 0x7fffffff;
        if (t) {
            bnmin = t->bnmin;
            if (np > 0) {
                W = t->units[np - 1];
                T = t->tiles[np - 1];
            }
            wmin = t->wmin;
            wmax = t->wmax;
        } else {
            bnmin = kTileN;
            for (int q = 0; q < np; ++q) {
                const MmaProb &pr = p[q];
                if (pr.tc_ntiles == 0 || !tile_active(pr.st)) continue;
                bnmin = tile_bn(pr) < bnmin ? tile_bn(pr) : bnmin;
            }
            for (int q = 0; q < np; ++q) {
                const MmaProb &pr = p[q];
                if (pr.tc_ntiles == 0 || !tile_active(pr.st)) continue;
                const int w = tile_units(pr);
                W += static_cast<long long>(pr.tc_ntiles) * w;
                T += pr.tc_ntiles;
                wmax = w > wmax ? w : wmax;
                wmin = w < wmin ? w : wmin;
            }
        }
        const long long grid = gridDim.x;
        const long long b = blockIdx.x;
        long long D = 0;  // tiles in whole data-parallel waves
        if (T > 0 && wmin == wmax && T >= 2 * grid) D = (T % grid == 0) ? T : (T / grid - 1) * grid;
        dp = b;
        dp_end = D;
        const long long Wsk = W - D * wmax;
        long long G = Wsk / wmax;
        if (G > grid) G = grid;
        if (G < 1) G = 1;
        if (Wsk <= 0 || b >= G) {
            g = end = 0;
        } else {
            g = D * wmax + Wsk * b / G;
            end = D * wmax + Wsk * (b + 1) / G;
        }
    }

    __device__ bool next(Seg &sg) {
        if (dp < dp_end) {
            long long r = dp;
            dp += gridDim.x;
            const int q = find(r, true);
            if (q < nprobs) {
                const MmaProb &pr = probs[q];
                sg.tile = pr.tc_tile0 + static_cast<int>(r);
                sg.prob = q;
                sg.k0 = 0;
                sg.nch = (step_chunks(pr.st, pr.n) > 0) ? tile_chunks(pr) : 0;
                sg.split = false;
                sg.head = true;
                return true;
            }
            dp = dp_end;
        }
        while (g < end) {
            long long r = g;
            const int q = find(r, false);
            if (q == nprobs) break;
            const MmaProb &pr = probs[q];
            const int f = unit_f(pr);
            const int w = tab ? tab->w[q] : tile_units(pr);
            const int nkc = w / f;
            const int ku = static_cast<int>(r % w);   // first unit of this range in the tile
            const long long left = end - g;
            const int k1u = (left < w - ku) ? ku + static_cast<int>(left) : w;
            g += k1u - ku;
            const int k = (ku + f - 1) / f, k1 = (k1u + f - 1) / f;  // chunks starting in [ku, k1u)
            if (k == k1) continue;
            sg.tile = pr.tc_tile0 + static_cast<int>(r / w);
            sg.prob = q;
            sg.k0 = k;
            sg.nch = (step_chunks(pr.st, pr.n) > 0) ? k1 - k : 0;
            sg.split = (k > 0) || (k1 < nkc);
            sg.head = (k == 0);
            return true;
        }
        g = end;
        return false;
    }
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait for a flag that a running CTA sets; false after limit_ns.
__device__ __forceinline__ bool flag_wait_bounded(const int *f, uint64_t limit_ns) {
    if (ld_acquire(f)) return true;
    const uint64_t t0 = globaltimer();
    while (!ld_acquire(f)) {
        if (globaltimer() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
    return true;
}

}  // namespace

__global__ void __launch_bounds__(kSymThreads, 1)
    k_sym_mma(const MmaProb *__restrict__ probs, int nprobs, const TileEnt *__restrict__ tiles,
              int ntiles, DevCtl *ctl, float *ws, int *cnt) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base_u32 = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
    StageSmem *stages = reinterpret_cast<StageSmem *>(smem);
    MmaSmemTail *tail = reinterpret_cast<MmaSmemTail *>(smem + sizeof(StageSmem) * kStages);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t wait_ns = ctl->wait_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&tail->full[s], 1);
            mbar_init(&tail->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tail->cfull[a], 1);
            mbar_init(&tail->cempty[a], kEpiWarps);
        }
        tail->abort_flag = 0;
        fence_barrier_init();
    }
    // (one problem: its table entry is read directly)
    const SchedTab *tab = (nprobs > 1 && nprobs <= kSchedProbs) ? &tail->sch : nullptr;
    if (tab) sched_pass1(&tail->sch, probs, nprobs);
    if (warp == 1) tmem_alloc(&tail->tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tab) {
        if (warp == 0) sched_pass2(&tail->sch, nprobs, lane);
        __syncthreads();
    }
    const uint32_t tmem_base = tail->tmem_base;

    if (warp < kSymEpiWarp0) setmaxnreg_dec<kSymRegsLow>();
    if (warp == 0) {
        // ------------------------------------------------------------ producer
        uint32_t stage = 0, phase = 0;
        bool ok = true;
        uint32_t last_phase[kStages];
        bool issued[kStages];
        for (int s = 0; s < kStages; ++s) { issued[s] = false; last_phase[s] = 0; }
        SegIter it;
        it.init(probs, nprobs, tab);
        Seg sg;
        while (ok && it.next(sg)) {
            if (sg.tile >= ntiles) break;
            const TileEnt te = tiles[sg.tile];
            const MmaProb &pr = probs[sg.prob];
            const SolveState *st = pr.st;
            const int S = step_slices(st);
            const MatSlot &ma = pr.mats[st->op.A];
            const MatSlot &mb = pr.mats[st->op.B];
            const bool wide = tile_bn(pr) == kTileN;
            const CUtensorMap *tmb = wide ? mb.tmB : mb.tmA;  // B panel: 256 or 128 rows
            const uint32_t bytes = static_cast<uint32_t>(S * (kSliceABytes + (wide ? kSliceBBytes : kSliceABytes)));
            for (int kc = sg.k0; kc < sg.k0 + sg.nch; ++kc) {
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
                    for (int s = 0; s < S; ++s) {
                        tma_load_2d(stages[stage].a[s], &ma.tmA[s], &tail->full[stage],
                                    kc * kTileK, te.I * kTileM);
                        tma_load_2d(stages[stage].b[s], &tmb[s], &tail->full[stage],
                                    kc * kTileK, te.Jp * (wide ? kTileN : kTileM));
                    }
                }
                __syncwarp();
                issued[stage] = true;
                last_phase[stage] = phase;
                if (++stage == kStages) { stage = 0; phase ^= 1u; }
            }
        }
        if (!ok) {
            // no TMA write may still be in flight when the CTA exits; the last
            // phase issued on a stage is its newest, so waiting on it is exact
            tail->abort_flag = 1;
            if (lane == 0)
                for (int s = 0; s < kStages; ++s)
                    if (issued[s]) (void)mbar_wait_bounded(&tail->full[s], last_phase[s], wait_ns);
            __syncwarp();
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        uint32_t stage = 0, phase = 0;
        uint32_t chunk = 0;  // chunk counter of this CTA: buffer = chunk & 1
        bool ok = true;
        bool any_commit = false;
        constexpr uint32_t idesc_w = idesc_f16(kTileM, kTileN, 0);
        constexpr uint32_t idesc_n = idesc_f16(kTileM, kTileM, 0);
        SegIter it;
        it.init(probs, nprobs, tab);
        Seg sg;
        while (ok && it.next(sg)) {
            if (sg.tile >= ntiles) break;
            const TileEnt te = tiles[sg.tile];
            const MmaProb &pr = probs[sg.prob];
            const SolveState *st = pr.st;
            const int S = step_slices(st);
            const uint32_t idesc = (tile_bn(pr) == kTileN) ? idesc_w : idesc_n;
            for (int kc = sg.k0; kc < sg.k0 + sg.nch; ++kc) {
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
                    const uint32_t tmem_d = tmem_base + buf * kTileN;
                    const uint64_t a0 = smem_desc_sw128(stages[stage].a[0]);
                    const uint64_t b0 = smem_desc_sw128(stages[stage].b[0]);
                    uint32_t accum = 0;
                    if (S == 2) {
                        const uint64_t a1 = smem_desc_sw128(stages[stage].a[1]);
                        const uint64_t b1 = smem_desc_sw128(stages[stage].b[1]);
                        // small cross terms first: hi * lo, lo * hi
#pragma unroll
                        for (int kk = 0; kk < kTileK / 16; ++kk) {
                            const uint64_t off = static_cast<uint64_t>(kk * 2);  // 32 B along K
                            tc_mma_f16(tmem_d, a0 + off, b1 + off, idesc, accum);
                            accum = 1;
                            tc_mma_f16(tmem_d, a1 + off, b0 + off, idesc, accum);
                        }
                    }
                    // the full-magnitude hi * hi terms last
#pragma unroll
                    for (int kk = 0; kk < kTileK / 16; ++kk) {
                        const uint64_t off = static_cast<uint64_t>(kk * 2);
                        tc_mma_f16(tmem_d, a0 + off, b0 + off, idesc, accum);
                        accum = 1;
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
            tail->abort_flag = 1;
            // every issued MMA must finish before TMEM is released
            if (lane == 0 && any_commit) {
                uint64_t *drain = &tail->cfull[chunk & 1u];
                tc_commit(drain);
                (void)mbar_wait_bounded(drain, (chunk >> 1) & 1u, wait_ns);
            }
            __syncwarp();
        }
    } else if (warp >= kSymEpiWarp0) {
        // ------------------------------------------------------------ drain + epilogue
        setmaxnreg_inc<kSymRegsHigh>();
        const int ew = warp - kSymEpiWarp0;    // 0..7
        const int q = warp & 3;                // TMEM lane quadrant (hardware rule: warp % 4)
        const int h = ew >> 2;                 // column half of the tile
        const int row_local = q * 32 + lane;
        uint32_t chunk = 0;
        bool ok = true;
        SegIter it;
        it.init(probs, nprobs, tab);
        Seg sg;
        while (ok && it.next(sg)) {
            if (sg.tile >= ntiles) break;
            const TileEnt te = tiles[sg.tile];
            const MmaProb &pr = probs[sg.prob];
            const SolveState *st = pr.st;
            const int n = pr.n;
            const bool wide = tile_bn(pr) == kTileN;
            const int ncol = wide ? 128 : 64;  // columns of this warp's strip
            float acc[128];
#pragma unroll
            for (int c = 0; c < 128; ++c) acc[c] = 0.0f;
            for (int kc = sg.k0; kc < sg.k0 + sg.nch; ++kc) {
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
                const uint32_t tbase = tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                                       buf * kTileN + static_cast<uint32_t>(h * ncol);
#pragma unroll
                for (int c2 = 0; c2 < 2; ++c2) {
                    if (c2 * 64 < ncol) {
                        float v[64];
                        tmem_ld64(tbase + c2 * 64, v);
#pragma unroll
                        for (int u = 0; u < 64; ++u) acc[c2 * 64 + u] += v[u];
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tail->cempty[buf]);
                ++chunk;
            }
            // a warp leaves the chunk loop early only on a timeout; make the
            // decision uniform over the drain warps before the named barriers
            if (lane == 0) tail->vote[ew] = ok ? 1 : 0;
            epi_bar();
            bool all_ok = true;
            for (int w = 0; w < kEpiWarps; ++w) all_ok = all_ok && (tail->vote[w] != 0);
            epi_bar();
            if (!all_ok) {
                ok = false;
                break;
            }

            // ---- a tile shared with a neighbouring CTA: the first to arrive
            // hands its partial sums over through global memory, the second
            // adds them (one commutative addition: the same result whoever is
            // second) and runs the epilogue.  The second waits only for a CTA
            // that is already writing, so the wait is short and bounded.
            if (sg.split) {
                const int slot = sg.head ? static_cast<int>(blockIdx.x) : static_cast<int>(blockIdx.x) - 1;
                float4 *wsp = reinterpret_cast<float4 *>(ws + static_cast<size_t>(slot) * kSkSlotFloats +
                                                         (static_cast<size_t>(ew) * 32 + lane) * 128);
                if (ew == 0 && lane == 0) tail->sk_ticket = atomicAdd(&cnt[2 * slot], 1);
                epi_bar();
                const int ticket = tail->sk_ticket;
                epi_bar();
                if (ticket == 0) {
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        if (4 * c < ncol)
                            wsp[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                    __threadfence();
                    epi_bar();
                    if (ew == 0 && lane == 0) atomicExch(&cnt[2 * slot + 1], 1);
                    continue;
                }
                if (ew == 0 && lane == 0) {
                    const int *flag = ctl->fail_partner ? &ctl->never : &cnt[2 * slot + 1];
                    tail->sk_ok = flag_wait_bounded(flag, wait_ns) ? 1 : 0;
                }
                epi_bar();
                const bool got = tail->sk_ok != 0;
                epi_bar();
                if (!got) {
                    if (ew == 0 && lane == 0) record_error(ctl, kErrTimeoutPartner);
                    ok = false;
                    break;
                }
                __threadfence();
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    if (4 * c >= ncol) break;
                    const float4 p4 = __ldcg(wsp + c);
                    acc[4 * c] += p4.x;
                    acc[4 * c + 1] += p4.y;
                    acc[4 * c + 2] += p4.z;
                    acc[4 * c + 3] += p4.w;
                }
                epi_bar();
                if (ew == 0 && lane == 0) {
                    atomicExch(&cnt[2 * slot], 0);
                    atomicExch(&cnt[2 * slot + 1], 0);
                }
            }

            // ---- store phase for the strip of block J (J = 2 Jp + h when bn =
            // 256, else J = Jp and columns 64 h .. 64 h + 63 of it)
            // Lane = row i of the warp's 32-row strip.  The masters E1/E2 are
            // symmetric, so they are read at (j, i): lanes on consecutive
            // addresses.  Mirrored writes (j, i) are coalesced the same way;
            // direct writes (i, j) go through a per-warp staging buffer so that
            // each store instruction covers 4 rows x 8 consecutive columns.
            // Columns are taken 8 at a time.  E1/E2 are re-read per output (L1
            // hits): the control kernel lets an output overwrite E1/E2 in place
            // only when it is the step's single output.
            const ProdOp &op = st->op;
            const float inv = op.inv;
            const int ldy = pr.ldy, lds = pr.lds, ldx = pr.ldx;
            const float *E1 = (op.E1 >= 0) ? pr.mats[op.E1].master : nullptr;
            const float *E2 = (op.E2 >= 0) ? pr.mats[op.E2].master : nullptr;
            const int nout = op.nout, pout = op.part_out;
            const float ra = op.ra, rb = op.rb, rc = op.rc;
            if (lane < nout) {
                const OutSpec &o = op.out[lane];
                OutCache &c = tail->oc[ew][lane];
                c.a = o.a;
                c.b1 = o.b1;
                c.b2 = o.b2;
                c.s = o.s;
                c.g1r = o.g1r;
                c.g1c = o.g1c;
                c.g2r = o.g2r;
                c.g2c = o.g2c;
                c.flags = o.flags;
                c.master = pr.mats[o.mat].master;
                c.sl0 = pr.mats[o.mat].sl[0];
                c.sl1 = pr.mats[o.mat].sl[1];
            }
            __syncwarp();
            const int i0 = te.I * kTileM + q * 32;
            const int i = i0 + lane;
            const int J = wide ? 2 * te.Jp + h : te.Jp;
            const int cb = J * kTileM + (wide ? 0 : 64 * h);  // first column of the strip
            const int ng = ncol / 8;                            // its 8-column groups
            double tr = 0.0, sq = 0.0, tr1 = 0.0, rr = 0.0;
            double *stg = tail->stage[ew];
            float *stf = reinterpret_cast<float *>(stg);
            const int rsub = lane >> 3, csub = lane & 7;  // direct-write lane layout
            const bool lean = nout == 1 && pout == 0 && !E2 && op.out[0].flags == (kOutMaster | kOutSlices);
            if (lean && J >= te.I && cb < n && i0 < n) {
                // the zero-temperature step: one output a v + b1 E1 + c [i == j].
                // An 8-column group wholly inside the matrix and above the
                // diagonal (every element exists and counts twice) takes the
                // vector path: each lane reads E1 and writes its own row's 8
                // columns with 16-byte accesses, and the mirrored rows go
                // through the staging buffer (layout [column][row], stride 33:
                // conflict-free both ways) so that 4 lanes write 8 consecutive
                // elements each of one row.  Other groups (the diagonal's, the
                // matrix edge) take the element-wise path.
                const bool diag = (J == te.I);
                const OutSpec &os = op.out[0];
                const MatSlot &m = pr.mats[os.mat];
                const float oa = os.a, ob = os.b1, oc = static_cast<float>(os.c), osc = os.s;
                float *Mo = m.master;
                __half *S0 = m.sl[0], *S1 = m.sl[1];
                const int mr = lane >> 2;        // mirrored row within the group
                const int mc = (lane & 3) * 8;   // its first column within the strip
                // a group takes the vector path when all of it exists and lies
                // above the diagonal; its E1 row segment is loaded one group
                // ahead, so the load's latency overlaps the previous group
                auto vec_group = [&](int c) {
                    const int jc = cb + c * 8;
                    return i0 + 32 <= n && jc + 8 <= n && (!diag || jc >= i0 + 32);
                };
                float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
                if (vec_group(0)) {
                    const size_t r0 = static_cast<size_t>(i) * ldy + cb;
                    pa = *reinterpret_cast<const float4 *>(E1 + r0);
                    pb = *reinterpret_cast<const float4 *>(E1 + r0 + 4);
                }
#pragma unroll
                for (int c8 = 0; c8 < kTileM / 8; ++c8) {
                    const int j0 = cb + c8 * 8;
                    if (c8 >= ng || j0 >= n) break;
                    const float4 ea = pa, eb = pb;  // this group's E1 (when it is a vector group)
                    if (c8 + 1 < ng && vec_group(c8 + 1)) {
                        const size_t rn = static_cast<size_t>(i) * ldy + j0 + 8;
                        pa = *reinterpret_cast<const float4 *>(E1 + rn);
                        pb = *reinterpret_cast<const float4 *>(E1 + rn + 4);
                    }
                    if (diag && j0 + 7 < i0) continue;
                    const bool full = vec_group(c8);
                    if (full) {
                        const size_t ro = static_cast<size_t>(i) * ldy + j0;
                        const float e[8] = {ea.x, ea.y, ea.z, ea.w, eb.x, eb.y, eb.z, eb.w};
                        float val[8];
                        float csq = 0.0f, crr = 0.0f;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float v = acc[c8 * 8 + u] * inv;
                            val[u] = fmaf(oa, v, ob * e[u]);
                            const float r = fmaf(ra, v, rb * e[u]);
                            csq = fmaf(val[u], val[u], csq);
                            crr = fmaf(r, r, crr);
                            stf[u * 33 + lane] = val[u];
                        }
                        sq += 2.0 * static_cast<double>(csq);
                        rr += 2.0 * static_cast<double>(crr);
                        *reinterpret_cast<float4 *>(Mo + ro) = make_float4(val[0], val[1], val[2], val[3]);
                        *reinterpret_cast<float4 *>(Mo + ro + 4) = make_float4(val[4], val[5], val[6], val[7]);
                        uint4 hv, lv;
                        split8(val, osc, hv, lv);
                        const size_t so = static_cast<size_t>(i) * lds + j0;
                        *reinterpret_cast<uint4 *>(S0 + so) = hv;
                        *reinterpret_cast<uint4 *>(S1 + so) = lv;
                        __syncwarp();
                        float w[8];
#pragma unroll
                        for (int t2 = 0; t2 < 8; ++t2) w[t2] = stf[mr * 33 + mc + t2];
                        __syncwarp();
                        const size_t mo = static_cast<size_t>(j0 + mr) * ldy + i0 + mc;
                        *reinterpret_cast<float4 *>(Mo + mo) = make_float4(w[0], w[1], w[2], w[3]);
                        *reinterpret_cast<float4 *>(Mo + mo + 4) = make_float4(w[4], w[5], w[6], w[7]);
                        split8(w, osc, hv, lv);
                        const size_t ms = static_cast<size_t>(j0 + mr) * lds + i0 + mc;
                        *reinterpret_cast<uint4 *>(S0 + ms) = hv;
                        *reinterpret_cast<uint4 *>(S1 + ms) = lv;
                        continue;
                    }
                    float csq = 0.0f, crr = 0.0f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = j0 + u;
                        float val = 0.0f;
                        if (i < n && j < n && (!diag || j >= i)) {
                            const bool on_diag = (j == i);
                            const size_t mt = static_cast<size_t>(j) * ldy + i;
                            const float v = acc[c8 * 8 + u] * inv;
                            const float e1 = E1 ? E1[mt] : 0.0f;
                            val = fmaf(oa, v, ob * e1) + (on_diag ? oc : 0.0f);
                            const float r = fmaf(ra, v, rb * e1) + (on_diag ? rc : 0.0f);
                            if (!on_diag) {
                                Mo[mt] = val;
                                const float ys = val * osc;
                                const __half hh = __float2half_rn(ys);
                                const size_t ms = static_cast<size_t>(j) * lds + i;
                                S0[ms] = hh;
                                S1[ms] = __float2half_rn(ys - __half2float(hh));
                            } else {
                                tr += static_cast<double>(val);
                            }
                            csq = fmaf(on_diag ? val : 2.0f * val, val, csq);
                            crr = fmaf(on_diag ? r : 2.0f * r, r, crr);
                        }
                        stf[lane * 9 + u] = val;
                    }
                    sq += static_cast<double>(csq);
                    rr += static_cast<double>(crr);
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int ii = i0 + 4 * k + rsub, jj = j0 + csub;
                        if (ii < n && jj < n && (!diag || jj >= ii)) {
                            const float val = stf[(4 * k + rsub) * 9 + csub];
                            Mo[static_cast<size_t>(ii) * ldy + jj] = val;
                            const float ys = val * osc;
                            const __half hh = __float2half_rn(ys);
                            const size_t ms = static_cast<size_t>(ii) * lds + jj;
                            S0[ms] = hh;
                            S1[ms] = __float2half_rn(ys - __half2float(hh));
                        }
                    }
                    __syncwarp();
                }
            } else if (J >= te.I && cb < n && i0 < n) {
                // any other step (1-3 outputs, E1/E2, FP64 outputs): groups
                // wholly above the diagonal take the 16-byte path as in the
                // zero-temperature step (one output after another; an output
                // overwrites E1/E2 in place only when it is the single one)
                const bool diag = (J == te.I);
                bool has_f64 = false;
                for (int o = 0; o < nout; ++o) has_f64 = has_f64 || (op.out[o].flags & (kOutF64a | kOutF64b));
                // diagonal form: the outputs of one step share their E1 / E2
                // coefficient vectors (the control kernel sets them so); the
                // row's entries are read once per strip, the columns' once per group
                int ev1 = -1, ev2 = -1;
                for (int o = 0; o < nout; ++o) {
                    if (!(op.out[o].flags & kOutDiag)) continue;
                    if (op.out[o].v1 >= 0) ev1 = op.out[o].v1;
                    if (op.out[o].v2 >= 0) ev2 = op.out[o].v2;
                }
                bool dup = false;  // a diagonal-form step: its masters are upper-triangular
                for (int o = 0; o < nout; ++o) dup = dup || (op.out[o].flags & kOutDiag);
                const float *F1 = (ev1 >= 0) ? pr.dgf[ev1] : nullptr;
                const float *F2 = (ev2 >= 0) ? pr.dgf[ev2] : nullptr;
                const float d1i = (F1 && i < n) ? F1[i] : 0.0f;
                const float d2i = (F2 && i < n) ? F2[i] : 0.0f;
                const int mr = lane >> 2, mc = (lane & 3) * 8;
#pragma unroll
                for (int c8 = 0; c8 < kTileM / 8; ++c8) {
                    const int j0 = cb + c8 * 8;
                    if (c8 >= ng || j0 >= n) break;
                    if (diag && j0 + 7 < i0) continue;  // strictly below the diagonal
                    if (!has_f64 && i0 + 32 <= n && j0 + 8 <= n && (!diag || j0 >= i0 + 32)) {
                        const size_t ro = static_cast<size_t>(i) * ldy + j0;
                        float e1[8], e2[8], v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) { e1[u] = 0.0f; e2[u] = 0.0f; }
                        if (E1) {
                            const float4 a4 = *reinterpret_cast<const float4 *>(E1 + ro);
                            const float4 b4 = *reinterpret_cast<const float4 *>(E1 + ro + 4);
                            e1[0] = a4.x; e1[1] = a4.y; e1[2] = a4.z; e1[3] = a4.w;
                            e1[4] = b4.x; e1[5] = b4.y; e1[6] = b4.z; e1[7] = b4.w;
                        }
                        if (E2) {
                            const float4 a4 = *reinterpret_cast<const float4 *>(E2 + ro);
                            const float4 b4 = *reinterpret_cast<const float4 *>(E2 + ro + 4);
                            e2[0] = a4.x; e2[1] = a4.y; e2[2] = a4.z; e2[3] = a4.w;
                            e2[4] = b4.x; e2[5] = b4.y; e2[6] = b4.z; e2[7] = b4.w;
                        }
                        float crr = 0.0f;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            v[u] = acc[c8 * 8 + u] * inv;
                            const float r = fmaf(ra, v[u], rb * e1[u]);
                            crr = fmaf(r, r, crr);
                        }
                        rr += 2.0 * static_cast<double>(crr);
                        const size_t so = static_cast<size_t>(i) * lds + j0;
                        const size_t mo = static_cast<size_t>(j0 + mr) * ldy + i0 + mc;
                        const size_t ms = static_cast<size_t>(j0 + mr) * lds + i0 + mc;
                        for (int o = 0; o < nout; ++o) {
                            const OutCache &os = tail->oc[ew][o];
                            const int fl = os.flags;
                            float val[8];
                            float csq = 0.0f;
                            if (fl & kOutDiag) {
                                // per-row / per-column coefficients of E1 and E2
                                const float r1 = fmaf(os.g1r, d1i, os.b1);
                                const float r2 = fmaf(os.g2r, d2i, os.b2);
#pragma unroll
                                for (int u = 0; u < 8; u += 4) {
                                    // FP32 copies, 32-byte aligned (j0 % 8 == 0, stride % 8 == 0)
                                    const float4 f1 = F1 ? *reinterpret_cast<const float4 *>(F1 + j0 + u)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                                    const float4 f2 = F2 ? *reinterpret_cast<const float4 *>(F2 + j0 + u)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                                    val[u] = fmaf(os.a, v[u], fmaf(fmaf(os.g1c, f1.x, r1), e1[u], fmaf(os.g2c, f2.x, r2) * e2[u]));
                                    val[u + 1] = fmaf(os.a, v[u + 1],
                                                      fmaf(fmaf(os.g1c, f1.y, r1), e1[u + 1], fmaf(os.g2c, f2.y, r2) * e2[u + 1]));
                                    val[u + 2] = fmaf(os.a, v[u + 2],
                                                      fmaf(fmaf(os.g1c, f1.z, r1), e1[u + 2], fmaf(os.g2c, f2.z, r2) * e2[u + 2]));
                                    val[u + 3] = fmaf(os.a, v[u + 3],
                                                      fmaf(fmaf(os.g1c, f1.w, r1), e1[u + 3], fmaf(os.g2c, f2.w, r2) * e2[u + 3]));
                                }
                            } else {
#pragma unroll
                                for (int u = 0; u < 8; ++u) val[u] = fmaf(os.a, v[u], fmaf(os.b1, e1[u], os.b2 * e2[u]));
                            }
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                csq = fmaf(val[u], val[u], csq);
                                stf[u * 33 + lane] = val[u];
                            }
                            if (o == pout) sq += 2.0 * static_cast<double>(csq);
                            uint4 hv, lv;
                            if (fl & kOutMaster) {
                                *reinterpret_cast<float4 *>(os.master + ro) = make_float4(val[0], val[1], val[2], val[3]);
                                *reinterpret_cast<float4 *>(os.master + ro + 4) = make_float4(val[4], val[5], val[6], val[7]);
                            }
                            if (fl & kOutSlices) {
                                split8(val, os.s, hv, lv);
                                *reinterpret_cast<uint4 *>(os.sl0 + so) = hv;
                                *reinterpret_cast<uint4 *>(os.sl1 + so) = lv;
                            }
                            __syncwarp();
                            float w[8];
#pragma unroll
                            for (int t2 = 0; t2 < 8; ++t2) w[t2] = stf[mr * 33 + mc + t2];
                            __syncwarp();
                            if ((fl & kOutMaster) && !(fl & kOutDiag)) {  // diagonal form: upper master only
                                *reinterpret_cast<float4 *>(os.master + mo) = make_float4(w[0], w[1], w[2], w[3]);
                                *reinterpret_cast<float4 *>(os.master + mo + 4) = make_float4(w[4], w[5], w[6], w[7]);
                            }
                            if (fl & kOutSlices) {
                                split8(w, os.s, hv, lv);
                                *reinterpret_cast<uint4 *>(os.sl0 + ms) = hv;
                                *reinterpret_cast<uint4 *>(os.sl1 + ms) = lv;
                            }
                        }
                        continue;
                    }
                    // element (i, j0 + u) exists in this block's upper part
                    auto okf = [&](int u) { return i < n && j0 + u < n && (!diag || j0 + u >= i); };
                    // E masters of a diagonal-form step hold the upper triangle only
                    // (read at (i, j)); others are read at (j, i), lanes on
                    // consecutive addresses
                    auto e_at = [&](int u) {
                        return dup ? static_cast<size_t>(i) * ldy + j0 + u : static_cast<size_t>(j0 + u) * ldy + i;
                    };
                    auto e1f = [&](int u) { return E1 ? E1[e_at(u)] : 0.0f; };
                    auto e2f = [&](int u) { return E2 ? E2[e_at(u)] : 0.0f; };
                    // off-diagonal value of an output (diagonal form: per-row and
                    // per-column E coefficients)
                    auto offv = [&](const OutSpec &os, int u) -> float {
                        const float vv = acc[c8 * 8 + u] * inv;
                        if (!(os.flags & kOutDiag)) return fmaf(os.a, vv, fmaf(os.b1, e1f(u), os.b2 * e2f(u)));
                        const int j = j0 + u;
                        const float c1 = os.b1 + os.g1r * d1i + (F1 ? os.g1c * F1[j] : 0.0f);
                        const float c2 = os.b2 + os.g2r * d2i + (F2 ? os.g2c * F2[j] : 0.0f);
                        return fmaf(os.a, vv, fmaf(c1, e1f(u), c2 * e2f(u)));
                    };
                    // diagonal entry of an output in the diagonal form, FP64
                    auto diagv = [&](const OutSpec &os, int u) -> double {
                        double r = os.c + static_cast<double>(os.a) * static_cast<double>(acc[c8 * 8 + u] * inv);
                        const double dxv = (os.dx >= 0) ? pr.dg[os.dx][i] : 0.0;
                        const double dyv = (os.dy >= 0) ? pr.dg[os.dy][i] : 0.0;
                        return r + os.q * dxv * dyv + os.l1 * dxv + os.l2 * dyv;
                    };
                    float crr = 0.0f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (okf(u)) {
                            const bool on_diag = (j0 + u == i);
                            const float r = fmaf(ra, acc[c8 * 8 + u] * inv, rb * e1f(u)) + (on_diag ? rc : 0.0f);
                            crr = fmaf(on_diag ? r : 2.0f * r, r, crr);
                        }
                    }
                    rr += static_cast<double>(crr);
                    for (int o = 0; o < nout; ++o) {
                        const OutSpec &os = op.out[o];
                        const int fl = os.flags;
                        if (fl & (kOutF64a | kOutF64b)) {
                            double *X = pr.Xd[(fl & kOutF64a) ? 0 : 1];
                            const double *Xa = (fl & kOutF64Add) ? pr.Xd[(fl & kOutF64a) ? 1 : 0] : nullptr;
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int j = j0 + u;
                                const bool on_diag = (j == i);
                                double d = 0.0;
                                if (okf(u)) {
                                    // the FP32 terms summed in FP32 and converted exactly by
                                    // integer operations: GB300's FP64 pipe (1/64 of the FP32
                                    // rate) keeps only the FP64 diagonal, the FP64 addend and
                                    // the squared norm
                                    if ((fl & kOutDiag) && on_diag) {
                                        d = diagv(os, u);
                                    } else if (fl & kOutDiag) {
                                        d = f32_to_f64(offv(os, u));
                                    } else {
                                        d = f32_to_f64(fmaf(os.a, acc[c8 * 8 + u] * inv, fmaf(os.b1, e1f(u), os.b2 * e2f(u))));
                                        if (on_diag) d += os.c;
                                    }
                                    if (Xa) d += Xa[static_cast<size_t>(j) * ldx + i];  // symmetric: read at (j, i)
                                    if (!on_diag) X[static_cast<size_t>(j) * ldx + i] = d;
                                    if (o == pout) {
                                        if (on_diag) tr += d;
                                        sq = fma(on_diag ? d : 2.0 * d, d, sq);
                                    }
                                    if (o == 1 && on_diag) tr1 += d;
                                }
                                stg[lane * 9 + u] = d;
                            }
                            __syncwarp();
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const int ii = i0 + 4 * k + rsub, jj = j0 + csub;
                                if (ii < n && jj < n && (!diag || jj >= ii))
                                    X[static_cast<size_t>(ii) * ldx + jj] = stg[(4 * k + rsub) * 9 + csub];
                            }
                            __syncwarp();
                            continue;
                        }
                        const MatSlot &m = pr.mats[os.mat];
                        const float cdiag = static_cast<float>(os.c);
                        const bool dform = (fl & kOutDiag) != 0;
                        float csq = 0.0f;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int j = j0 + u;
                            const bool on_diag = (j == i);
                            float val = 0.0f;
                            if (okf(u)) {
                                if (dform && on_diag) {
                                    // the diagonal goes to the FP64 vector; the small part keeps 0
                                    const double dv = diagv(os, u);
                                    pr.dg[os.mat][i] = dv;
                                    pr.dgf[os.mat][i] = static_cast<float>(dv);
                                    if (o == pout) {
                                        tr += dv;
                                        sq += dv * dv;
                                    }
                                    if (o == 1) tr1 += dv;
                                } else {
                                    val = offv(os, u) + ((on_diag && !dform) ? cdiag : 0.0f);
                                    if (!on_diag) {
                                        if ((fl & kOutMaster) && !dform) m.master[static_cast<size_t>(j) * ldy + i] = val;
                                        if (fl & kOutSlices) put_slices(m, static_cast<size_t>(j) * lds + i, val * os.s);
                                    }
                                    if (o == pout) {
                                        if (on_diag) tr += static_cast<double>(val);
                                        csq = fmaf(on_diag ? val : 2.0f * val, val, csq);
                                    }
                                    if (o == 1 && on_diag) tr1 += static_cast<double>(val);
                                }
                            }
                            stf[lane * 9 + u] = val;
                        }
                        if (o == pout) sq += static_cast<double>(csq);
                        __syncwarp();
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int ii = i0 + 4 * k + rsub, jj = j0 + csub;
                            if (ii < n && jj < n && (!diag || jj >= ii)) {
                                const float val = stf[(4 * k + rsub) * 9 + csub];
                                if (fl & kOutMaster) m.master[static_cast<size_t>(ii) * ldy + jj] = val;
                                if (fl & kOutSlices) put_slices(m, static_cast<size_t>(ii) * lds + jj, val * os.s);
                            }
                        }
                        __syncwarp();
                    }
                }
            }
            // deterministic per-tile partials: warp tree, then the 8 warps in order
            tr = warp_sum(tr);
            sq = warp_sum(sq);
            tr1 = warp_sum(tr1);
            rr = warp_sum(rr);
            if (lane == 0) {
                tail->red[ew][0] = tr;
                tail->red[ew][1] = sq;
                tail->red[ew][2] = tr1;
                tail->red[ew][3] = rr;
            }
            epi_bar();
            if (ew == 0 && lane == 0) {
                double a = 0, b = 0, c = 0, d = 0;
                for (int w = 0; w < kEpiWarps; ++w) {
                    a += tail->red[w][0];
                    b += tail->red[w][1];
                    c += tail->red[w][2];
                    d += tail->red[w][3];
                }
                double *slot = pr.part + static_cast<size_t>(te.slot) * kPartStride;
                slot[0] = a;
                slot[1] = b;
                slot[2] = c;
                slot[3] = d;
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

size_t mma_smem_bytes() { return kMmaSmemBytes; }

}  // namespace fe
