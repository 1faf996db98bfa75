// Host side of the C ABI declared in include/fe.h and include/fe_kernels.h.
//
// A context owns one CUDA stream, an HBM-budgeted pool of per-problem "slots"
// (Hp copy, FP32 master, FP16 slice sets, FP64 buffers, partials, state), the
// launch sequences and the tile-shape table (tensor-core tile width per
// number of 128-row panels and precision policy, filled by the autotuners).  A solve (or a batch of solves) is:
//   bounds rows + reduce + X0 init              (per problem)
//   repeat:  control (1 block / problem)  ->  tensor-core step over the tiles
//            of all problems  ->  FP64 step over the 64x64 tiles of all
//            problems                      (kernels skip problems whose state
//                                             says the step is not theirs)
//   finalize (D out, tr(Hp D), tr D)            (per problem)
// with no host synchronisation until the end.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <climits>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/fe.h"
#include "../../include/fe_kernels.h"
#include "fe_dev.cuh"
#include "fe_kernels.cuh"

using namespace fe;

namespace {

// last failure of a call made by this thread (any context)
thread_local std::string g_err;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

struct Slot {
    int n = 0;
    int method = 0;  // kMethodSp2 / kMethodFermi: decides which matrices exist
    size_t bytes = 0;
    bool in_use = false;
    char *arena = nullptr;
    double *Hcopy = nullptr;
    float *Y = nullptr;
    double *Xd[2] = {};
    double *Dtmp = nullptr;
    float *lzv = nullptr;   // Lanczos vectors (3 n FP32)
    double *part = nullptr;
    SolveState *st = nullptr;
    RowInfo *rowinfo = nullptr;
    int *bad = nullptr;
    int ldy = 0, lds = 0, ldx = 0;
    std::vector<TileEnt> tiles;   // tensor-core tiles 128 x 256
    std::vector<TileEnt> tilesN;  // tensor-core tiles 128 x 128
    std::vector<Tile64> tiles64;
    std::vector<TileEnt> tilesD;  // digit-product tiles (zero temperature)
    MmaProb hp;  // host image of the device descriptor (H filled per solve)
};

// Launch state of one stream of work: device copies of the problem table and
// tile lists, pinned images of the solve states, error word, events.
struct Engine {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevCtl *d_err = nullptr;         // error word, wait limit and test hook of the kernels
    MmaProb *d_probs = nullptr;
    size_t probs_cap = 0;
    TileEnt *d_tiles = nullptr;
    size_t tiles_cap = 0;
    Tile64 *d_tiles64 = nullptr;
    size_t tiles64_cap = 0;
    TileEnt *d_tilesD = nullptr;
    std::vector<int> off64, cnt64;  // each problem's range in the FP64 tile list
    MmaProb *d_chk = nullptr;       // table of the problems certifying their bounds together
    size_t chk_cap = 0;
    size_t tilesD_cap = 0;
    SolveState *h_states = nullptr;  // pinned
    size_t h_states_cap = 0;
    int *h_done = nullptr;           // pinned copies of the done flags (serving)
    size_t h_done_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_setup = nullptr, ev_loop = nullptr;  // end of set-up, end of the step loop
    int ntc = 0, n64 = 0, nD = 0;    // tile counts of the uploaded lists
    bool any_tc = false, any_fp64 = false, any_digit = false;
    // the step loop as a CUDA graph: WHILE(any problem active) { IF(tc) k_sym_mma;
    // IF(fp64) k_fp64_step; IF(digit) k_digit_prep, k_digit_mma; k_control }
    StepFlags *d_flags = nullptr;
    StepFlags h_flags{};
    // Stream-K hand-off of split tiles in k_sym_mma: one slot and two counters per SM
    float *d_skws = nullptr;
    int *d_skcnt = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<uintptr_t> gkey;     // what the instantiated graph was built for
};

// One entry of the tile-shape table: the tensor-core tile width chosen for
// problems with a given number of 128-row panels under one precision policy,
// with the solve times (ms) the autotuner measured for each width (0: not
// measured, the entry was set directly).
struct TuneEnt {
    int bn = kTileN;
    double ms_w = 0.0, ms_n = 0.0;
};

// One fe_submit request.
struct Req {
    fe_ticket id = 0;
    fe_problem p{};                 // Hp points at hbuf (host) or at the slot's copy (device)
    std::vector<double> hbuf;       // host copy of Hp while no slot is free
    Slot *slot = nullptr;
    bool staged = false;            // Hp already copied into slot->Hcopy
    bool gershgorin = false;        // the spectral-bound estimate proved too tight: use Gershgorin
    bool accel_off = false;         // FE_METHOD_ASP2 estimates proved inconsistent: plain SP2
    bool deferred = false;          // waited at least once for a free part of the HBM budget
    int wasted = 0;                 // products of attempts that were started again
    int bn = 0;                     // tensor-core tile width, fixed when the solve starts
    bool done = false;
    fe_result res{};
    std::chrono::steady_clock::time_point t_submit;
};

}  // namespace

struct fe_ctx {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_iters = 100;
    uint32_t prec_default = FE_PREC_MIXED;
    int num_sms = 148;
    int lz_grid = 0;                 // blocks of the cooperative Lanczos launch (all resident)
    Engine eng;                      // blocking solves and batches
    std::mutex smu;                  // slots, used
    std::vector<Slot *> slots;
    // optional per-launch timing of the expansion kernels (fe_k_profile)
    bool prof = false;
    std::vector<cudaEvent_t> pev;
    double prof_out[8] = {};
    std::vector<double> prof_steps;  // tensor-core launch ms of each step of the last profiled solve
    double prof_kind_ms[8] = {};     // ... summed by the kind of step (first problem of the table)
    int prof_kind_n[8] = {};
    std::atomic<long long> launches{0};  // kernels launched by this context
    std::atomic<double> lz_narrow{1.0};  // test hook: scale of the estimated bound interval
    double phase_ms[4] = {};             // last blocking solve: set-up, step loop, output; steps
    // tile-shape table: (128-row panels, FE_PREC_*) -> tile width (fe_autotune)
    std::mutex tmu;
    std::map<std::pair<int, uint32_t>, TuneEnt> tune;
    std::string tune_path;               // file the table is loaded from / saved to ("" = none)
    std::recursive_mutex mu;  // eng, profiling state (blocking calls)
    // continuous batching (fe_submit / fe_poll): a worker thread with its own engine
    Engine seng;
    cudaStream_t copy_stream = nullptr;
    std::mutex qmu;
    std::condition_variable qcv;
    std::deque<Req *> waiting;       // submitted, not yet started
    std::map<fe_ticket, Req *> reqs; // every ticket not yet collected by fe_poll
    fe_ticket next_ticket = 1;
    std::thread worker;
    bool worker_started = false;
    bool stop = false;
    // serving counters (under qmu): requests submitted, requests that waited
    // for HBM at least once, largest queue of waiting requests, largest
    // number of requests on the device at once
    long long n_submitted = 0, n_deferred = 0;
    long long peak_waiting = 0, peak_running = 0;
    // fe_project / fe_rotate: FP16 slices of both operands and split-K
    // partial tiles (one arena, grown on demand), argument block, tile list
    char *gws = nullptr;
    size_t gws_cap = 0;
    GemmArgs *d_gargs = nullptr;
    TileEnt *d_gtiles = nullptr;
    size_t gtiles_cap = 0;
    unsigned long long *d_amax = nullptr;
};

namespace {

int set_err(fe_ctx *, int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(fe_ctx *ctx, cudaError_t e, const char *what) {
    return set_err(ctx, FE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FE_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Upper-triangle tiles (row panel I < nI, column panel jmin(I) <= J < nJ,
// jmin nondecreasing) in bands of `band` row panels, column by column within
// a band.  The product kernels hand out consecutive tiles to CTAs that run at
// the same time, so a wave then touches about `band` row panels and
// wave / band column panels instead of one or two rows of the triangle and
// every column.  `slot` stays the row-major index: per-tile partial sums land
// in the same places, and are reduced in the same order, whatever the order.
template <class Jmin>
void push_banded(std::vector<TileEnt> &out, int nI, int nJ, int band, Jmin jmin) {
    out.clear();
    std::vector<int> row0(nI + 1, 0);
    for (int I = 0; I < nI; ++I) row0[I + 1] = row0[I] + std::max(0, nJ - jmin(I));
    for (int b0 = 0; b0 < nI; b0 += band) {
        const int b1 = std::min(nI, b0 + band);
        for (int J = jmin(b0); J < nJ; ++J)
            for (int I = b0; I < b1; ++I)
                if (J >= jmin(I)) out.push_back(TileEnt{0, I, J, row0[I] + J - jmin(I)});
    }
}

// 128-row panels per band: the tensor-core tiles read 128 x K and 256 x K
// (or 128 x K) panels (two FP16 slices each), the digit tiles 128 x K and
// 64 x K panels of seven digits; the bands balance row-panel and column-panel
// bytes over a wave of about 150 tiles.
constexpr int kBandTc = 16, kBandTcN = 12, kBandDigit = 8;

void build_tiles(Slot *s) {
    const int T = ceil_div(s->n, kTileM);
    const int TP = ceil_div(T, 2);
    push_banded(s->tiles, T, TP, kBandTc, [](int I) { return I / 2; });
    push_banded(s->tilesN, T, T, kBandTcN, [](int I) { return I; });
    s->tiles64.clear();
    const int T64 = ceil_div(s->n, kTile64);
    int slot = 0;
    for (int I = 0; I < T64; ++I)
        for (int J = I; J < T64; ++J) s->tiles64.push_back(Tile64{0, I, J, slot++});
    s->tilesD.clear();
    if (s->method == kMethodSp2) {
        const int TD = ceil_div(s->n, kDigitN);
        push_banded(s->tilesD, T, TD, kBandDigit, [](int I) { return 2 * I; });
    }
}

// Matrices held per method: zero temperature keeps one FP32 master (Y) and two
// slice sets; finite temperature keeps masters for z, N, M, W, R and six slice
// sets (W has two, ping-pong, sharing one master).
int num_masters(int method) { return method == kMethodFermi ? 5 : 1; }
int num_slice_sets(int method) { return method == kMethodFermi ? kNumMats : 2; }

size_t slot_bytes(int n, int method, int *ldy, int *lds, int *ldx, size_t *nparts) {
    *ldy = static_cast<int>(align_up(n, 4));
    *lds = static_cast<int>(align_up(n, 8));
    *ldx = n;
    const int T = ceil_div(n, kTileM);
    const int T64 = ceil_div(n, kTile64);
    const size_t ntiles = static_cast<size_t>(T) * (T + 1) / 2;  // >= T ceil(T/2): either width
    const size_t nt64 = static_cast<size_t>(T64) * (T64 + 1) / 2;
    const size_t TD = static_cast<size_t>(ceil_div(n, kDigitN));
    size_t ntD = 0;
    for (size_t I = 0; I < static_cast<size_t>(T); ++I) ntD += (TD > 2 * I) ? TD - 2 * I : 0;
    *nparts = std::max<size_t>({static_cast<size_t>(kInitBlocks), ntiles, nt64, ntD,
                                static_cast<size_t>(kFinBlocks)});
    const size_t nn = static_cast<size_t>(n);
    size_t b = 0;
    auto add = [&](size_t x) { b += align_up(x, 1024); };
    add(8 * nn * nn);                                // Hcopy
    for (int k = 0; k < num_masters(method); ++k) add(4 * nn * (*ldy));  // FP32 masters
    for (int k = 0; k < num_slice_sets(method) * kMaxSlices; ++k) add(2 * nn * (*lds));  // slices
    add(8 * nn * (*ldx));                            // Xd[0]
    add(8 * nn * (*ldx));                            // Xd[1]
    add(8 * nn * nn);                                // Dtmp
    add(8 * 3 * nn);                                 // Lanczos vectors
    if (method == kMethodSp2)
        for (int a = 0; a < kDigits; ++a) add(2 * nn * (*lds));  // digits of X/4
    if (method == kMethodFermi) add(12 * kNumMats * align_up(nn, 8));  // FP64 diagonals + FP32 copies
    add(8 * kPartStride * (*nparts));                // partials
    add(sizeof(SolveState));
    add(sizeof(RowInfo) * nn);
    add(64);
    return b;
}

// A K-major FP16 operand of rows x kdim elements (leading dimension ld_elems),
// loaded in boxes of 64 (K) x box_rows with 128-byte swizzling.
int encode_map_rect(fe_ctx *ctx, CUtensorMap *m, void *base, int64_t kdim, int64_t rows, int64_t ld_elems,
                    int box_rows);

int encode_map(fe_ctx *ctx, CUtensorMap *m, void *base, int n, int ld_elems, int box_rows,
               int box_k = kTileK, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
    auto enc = get_encode();
    if (!enc) return set_err(ctx, FE_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(n)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld_elems) * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(box_k), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(ctx, FE_ECUDA, "cuTensorMapEncodeTiled failed");
    return FE_OK;
}

int encode_map_rect(fe_ctx *ctx, CUtensorMap *m, void *base, int64_t kdim, int64_t rows, int64_t ld_elems,
                    int box_rows) {
    auto enc = get_encode();
    if (!enc) return set_err(ctx, FE_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(kdim), static_cast<cuuint64_t>(rows)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld_elems) * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kTileK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(ctx, FE_ECUDA, "cuTensorMapEncodeTiled failed");
    return FE_OK;
}

void release_slot(fe_ctx *ctx, Slot *s) {
    std::lock_guard<std::mutex> lk(ctx->smu);
    s->in_use = false;
}

// caller holds ctx->smu
void free_slot(fe_ctx *ctx, Slot *s) {
    if (s->arena) cudaFree(s->arena);
    ctx->used -= s->bytes;
    delete s;
}

// A free slot for dimension n and method (reused if cached), or an error
// status with the error string set.
int acquire_slot(fe_ctx *ctx, int n, int method, Slot **out) {
    std::lock_guard<std::mutex> lk(ctx->smu);
    for (Slot *s : ctx->slots)
        if (!s->in_use && s->n == n && s->method == method) {
            s->in_use = true;
            *out = s;
            return FE_OK;
        }
    int ldy, lds, ldx;
    size_t nparts;
    const size_t bytes = slot_bytes(n, method, &ldy, &lds, &ldx, &nparts);
    if (bytes > ctx->budget)
        return set_err(ctx, FE_ENOMEM, "problem needs " + std::to_string(bytes) +
                                           " bytes, more than the HBM budget");
    // evict unused cached slots until it fits
    while (ctx->used + bytes > ctx->budget) {
        auto it = std::find_if(ctx->slots.begin(), ctx->slots.end(),
                               [](Slot *s) { return !s->in_use; });
        if (it == ctx->slots.end())
            return set_err(ctx, FE_ENOMEM, "HBM budget exhausted by active solves");
        Slot *v = *it;
        ctx->slots.erase(it);
        free_slot(ctx, v);
    }
    Slot *s = new Slot();
    s->n = n;
    s->method = method;
    s->bytes = bytes;
    s->ldy = ldy;
    s->lds = lds;
    s->ldx = ldx;
    cudaError_t e = cudaMalloc(&s->arena, bytes);
    if (e != cudaSuccess) {
        delete s;
        cudaGetLastError();
        return set_err(ctx, FE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ctx->used += bytes;
    const size_t nn = static_cast<size_t>(n);
    char *p = s->arena;
    auto take = [&](size_t x) {
        char *r = p;
        p += align_up(x, 1024);
        return r;
    };
    s->Hcopy = reinterpret_cast<double *>(take(8 * nn * nn));
    float *masters[5] = {};
    for (int k = 0; k < num_masters(method); ++k) masters[k] = reinterpret_cast<float *>(take(4 * nn * ldy));
    __half *slices[kNumMats][kMaxSlices] = {};
    for (int m = 0; m < num_slice_sets(method); ++m)
        for (int b = 0; b < kMaxSlices; ++b) slices[m][b] = reinterpret_cast<__half *>(take(2 * nn * lds));
    s->Y = masters[0];
    s->Xd[0] = reinterpret_cast<double *>(take(8 * nn * ldx));
    s->Xd[1] = reinterpret_cast<double *>(take(8 * nn * ldx));
    s->Dtmp = reinterpret_cast<double *>(take(8 * nn * nn));
    s->lzv = reinterpret_cast<float *>(take(4 * 3 * nn));
    __half *digs[kDigits] = {};
    if (method == kMethodSp2)
        for (int a = 0; a < kDigits; ++a) digs[a] = reinterpret_cast<__half *>(take(2 * nn * lds));
    const size_t dstride = align_up(nn, 8);  // 64-byte aligned vectors
    double *diags = (method == kMethodFermi) ? reinterpret_cast<double *>(take(12 * kNumMats * dstride)) : nullptr;
    s->part = reinterpret_cast<double *>(take(8 * kPartStride * nparts));
    s->st = reinterpret_cast<SolveState *>(take(sizeof(SolveState)));
    s->rowinfo = reinterpret_cast<RowInfo *>(take(sizeof(RowInfo) * nn));
    s->bad = reinterpret_cast<int *>(take(64));
    build_tiles(s);
    // descriptor image (tensor maps are fixed for the slot's lifetime)
    memset(&s->hp, 0, sizeof(MmaProb));
    for (int m = 0; m < num_slice_sets(method); ++m) {
        MatSlot &ms = s->hp.mats[m];
        for (int b = 0; b < kMaxSlices; ++b) {
            int rc = encode_map(ctx, &ms.tmA[b], slices[m][b], n, lds, kTileM);
            if (rc == FE_OK) rc = encode_map(ctx, &ms.tmB[b], slices[m][b], n, lds, kTileN);
            if (rc != FE_OK) {
                free_slot(ctx, s);
                return rc;
            }
            ms.sl[b] = slices[m][b];
        }
    }
    if (method == kMethodSp2) {
        for (int a = 0; a < kDigits; ++a) {
            const CUtensorMapSwizzle dswz = (kDigitK == 16) ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B;
            int rc = encode_map(ctx, &s->hp.dA[a], digs[a], n, lds, kTileM, kDigitK, dswz);
            if (rc == FE_OK)
                rc = encode_map(ctx, &s->hp.dB[a], digs[a], n, lds, kDigitN, kDigitK, dswz);
            if (rc != FE_OK) {
                free_slot(ctx, s);
                return rc;
            }
            s->hp.dig[a] = digs[a];
        }
    }
    if (method == kMethodFermi) {
        s->hp.mats[kMatZ].master = masters[0];
        s->hp.mats[kMatN].master = masters[1];
        s->hp.mats[kMatM].master = masters[2];
        s->hp.mats[kMatW0].master = masters[3];  // the two W slice sets share one master
        s->hp.mats[kMatW1].master = masters[3];
        s->hp.mats[kMatR].master = masters[4];
        float *diagf = reinterpret_cast<float *>(diags + kNumMats * dstride);
        for (int m = 0; m < kNumMats; ++m) {
            s->hp.dg[m] = diags + static_cast<size_t>(m) * dstride;
            s->hp.dgf[m] = diagf + static_cast<size_t>(m) * dstride;
        }
    } else {
        s->hp.mats[kMatY0].master = masters[0];  // both slice sets of Y share the master
        s->hp.mats[kMatY1].master = masters[0];
    }
    s->hp.Y = s->Y;
    s->hp.st = s->st;
    s->hp.part = s->part;
    s->hp.n = n;
    s->hp.ldy = ldy;
    s->hp.lds = lds;
    s->hp.ntiles = static_cast<int>(s->tiles.size());
    s->hp.bn = kTileN;
    s->hp.ntiles64 = static_cast<int>(s->tiles64.size());
    s->hp.ntilesD = static_cast<int>(s->tilesD.size());
    s->hp.lzv = s->lzv;
    s->hp.Xd[0] = s->Xd[0];
    s->hp.Xd[1] = s->Xd[1];
    s->hp.ldx = ldx;
    s->in_use = true;
    ctx->slots.push_back(s);
    *out = s;
    return FE_OK;
}

template <typename T>
int ensure_dev(fe_ctx *ctx, T **ptr, size_t *cap, size_t count) {
    if (count <= *cap) return FE_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    const size_t c = std::max<size_t>(count, 16);
    FE_CUDA(ctx, cudaMalloc(reinterpret_cast<void **>(ptr), sizeof(T) * c));
    *cap = c;
    return FE_OK;
}

uint32_t prec_of(const fe_ctx *ctx, const fe_problem *p) {
    uint32_t pr = p->flags & FE_PREC_MASK;
    if (pr == 0) pr = ctx->prec_default & FE_PREC_MASK;
    return pr;
}

// Tensor-core tile width for a problem of dimension n under precision policy
// prec: the table's entry for its number of 128-row panels, else the entry
// nearest in panels under the same policy, else 256.
int tile_width(fe_ctx *ctx, int64_t n, uint32_t prec) {
    const int T = static_cast<int>((n + kTileM - 1) / kTileM);
    std::lock_guard<std::mutex> lk(ctx->tmu);
    int best = kTileN, dist = INT_MAX;
    for (const auto &kv : ctx->tune) {
        if (kv.first.second != prec) continue;
        const int d = std::abs(kv.first.first - T);
        if (d < dist) {
            dist = d;
            best = kv.second.bn;
        }
    }
    return best;
}

// The expansion a problem runs (the solve state's method): FE_METHOD_ASP2 is
// the SP2 recursion with its folds switched on, FE_METHOD_TRFOE the truncated
// SP2 expansion at finite temperature.
int method_of(const fe_problem *p) {
    const uint32_t m = p->flags & FE_METHOD_MASK;
    if (m == FE_METHOD_TRFOE) return kMethodTrfoe;
    return (m == FE_METHOD_FERMI || (m == FE_METHOD_AUTO && p->kT > 0.0)) ? kMethodFermi : kMethodSp2;
}

// The buffers a problem's slot holds: the doubling recursion needs its own
// set; the SP2 forms (plain, accelerated, truncated) share one layout.
int slot_method(const fe_problem *p) { return method_of(p) == kMethodFermi ? kMethodFermi : kMethodSp2; }

// Step cap of the finite-temperature expansion: about 12 products per
// doubling (square, Newton-Schulz pairs, final product) for up to ~40
// doublings, plus the shift-only refinements.
constexpr int kFermiMaxSteps = 640;

int validate(fe_ctx *ctx, const fe_problem *p) {
    if (!p) return set_err(ctx, FE_EINVAL, "problem is NULL");
    if (!p->Hp) return set_err(ctx, FE_EINVAL, "Hp is NULL");
    if (p->n < 1 || p->n > (1 << 20)) return set_err(ctx, FE_EINVAL, "n out of range");
    if (p->ld < p->n) return set_err(ctx, FE_EINVAL, "ld < n");
    if (!(p->n_e >= 0.0) || p->n_e > static_cast<double>(p->n))
        return set_err(ctx, FE_EINVAL, "n_e outside [0, n]");
    if (!(p->kT >= 0.0) || !std::isfinite(p->kT)) return set_err(ctx, FE_EINVAL, "kT < 0");
    if (p->kT == 0.0 && p->n_e != std::floor(p->n_e))
        return set_err(ctx, FE_EINVAL, "non-integral n_e at kT == 0");
    if (!(p->tol >= 0.0)) return set_err(ctx, FE_EINVAL, "tol < 0");
    const uint32_t m = p->flags & FE_METHOD_MASK;
    if (m != FE_METHOD_AUTO && m != FE_METHOD_SP2 && m != FE_METHOD_FERMI && m != FE_METHOD_ASP2 &&
        m != FE_METHOD_TRFOE)
        return set_err(ctx, FE_EINVAL, "unknown method flag");
    if ((m == FE_METHOD_SP2 || m == FE_METHOD_ASP2) && p->kT != 0.0)
        return set_err(ctx, FE_EINVAL, "SP2 needs kT == 0");
    if (m == FE_METHOD_ASP2 && !(std::isfinite(p->homo) && std::isfinite(p->lumo) && p->homo < p->lumo))
        return set_err(ctx, FE_EINVAL, "FE_METHOD_ASP2 needs finite homo < lumo");
    if (m == FE_METHOD_TRFOE) {
        if (!(p->kT > 0.0)) return set_err(ctx, FE_EINVAL, "FE_METHOD_TRFOE needs kT > 0");
        const uint32_t pt = prec_of(ctx, p);
        if (pt != FE_PREC_MIXED && pt != FE_PREC_FP32 && pt != FE_PREC_FP64)
            return set_err(ctx, FE_EINVAL, "FE_METHOD_TRFOE runs FE_PREC_MIXED, FE_PREC_FP32 or FE_PREC_FP64");
    }
    const bool fermi = (m == FE_METHOD_FERMI) || (m == FE_METHOD_AUTO && p->kT > 0.0);
    if (fermi && !(p->kT > 0.0)) return set_err(ctx, FE_EINVAL, "FE_METHOD_FERMI needs kT > 0");
    const uint32_t pr = p->flags & FE_PREC_MASK;
    if (pr != FE_PREC_MIXED && pr != FE_PREC_FP64 && pr != FE_PREC_FP32 && pr != FE_PREC_TRY_FP16)
        return set_err(ctx, FE_EINVAL, "unknown precision flag");
    if (fermi && (prec_of(ctx, p) == FE_PREC_FP64 || prec_of(ctx, p) == FE_PREC_TRY_FP16))
        return set_err(ctx, FE_EINVAL, "the finite-temperature expansion runs split-FP16 products "
                                       "(FE_PREC_MIXED or FE_PREC_FP32)");
    if ((p->flags & ~(FE_PTR_DEVICE | FE_METHOD_MASK | FE_PREC_MASK)) != 0)
        return set_err(ctx, FE_EINVAL, "unknown flag bits");
    return FE_OK;
}

// Fill the pinned state image of one problem.
void init_state(const fe_ctx *ctx, const fe_problem *p, SolveState *st) {
    memset(st, 0, sizeof(SolveState));
    st->n = static_cast<int>(p->n);
    st->ne = p->n_e;
    st->kT = p->kT;
    st->tol = (p->tol > 0.0) ? p->tol : 5e-8;
    st->max_iters = ctx->max_iters;
    const uint32_t pr = prec_of(ctx, p);
    st->prec = (pr == FE_PREC_FP64) ? kPrecFp64
               : (pr == FE_PREC_FP32) ? kPrecFp32
               : (pr == FE_PREC_TRY_FP16) ? kPrecTryFp16 : kPrecMixed;
    st->phase = (st->prec == kPrecFp64) ? kPhaseFp64
                : (st->prec == kPrecTryFp16) ? kPhaseSingle : kPhaseSplit;
    st->kind = kNone;
    st->idem_hist[0] = st->idem_hist[1] = st->idem_hist[2] = DBL_MAX;
    st->fro_hist[0] = st->fro_hist[1] = st->fro_hist[2] = DBL_MAX;
    st->mu = NAN;
    st->method = method_of(p);
    if ((p->flags & FE_METHOD_MASK) == FE_METHOD_ASP2) {
        st->acc_on = 1;
        st->homo = p->homo;
        st->lumo = p->lumo;
    }
    if (st->method == kMethodTrfoe) {
        st->beta = 1.0 / p->kT;
        if (st->prec == kPrecTryFp16) st->prec = kPrecMixed;
    }
    if (st->method == kMethodFermi) {
        st->max_iters = kFermiMaxSteps;
        st->wcur = kMatW0;
        st->ft_sub = 0;  // x ready: the control starts with the tanh polynomial
    }
}
// ---------------------------------------------------------------- engine
// A set of problems on acquired slots runs as: eng_upload (problem table and
// tile lists of every problem in the set), eng_setup per newly started
// problem (Hp staging, state, bounds and X0 kernels, first control step),
// eng_steps (tensor-core step, FP64-accurate step, control step; repeated),
// eng_finish per finished problem (output kernels, read-back of its state).
// Kernels reach a problem's buffers and state through its table entry, so the
// table can be rebuilt between steps as problems join and leave; the tiles of
// one problem are computed the same way whatever else is in the table, so a
// problem's result does not depend on its batch.

// One problem bound to a slot.
struct Job {
    const fe_problem *p = nullptr;  // the caller's problem (D and its flag, n_e, kT, tol)
    Slot *slot = nullptr;
    const double *H = nullptr;      // device Hp the kernels read
    int64_t ldh = 0;
    const double *stage = nullptr;  // host Hp copied into slot->Hcopy at set-up, or null
    int64_t ldstage = 0;
    bool lanczos = true;            // estimate the spectral bounds (else Gershgorin)
    bool accel = true;              // FE_METHOD_ASP2: folds on (off after an inconsistent attempt)
    int bn = 0;                     // tensor-core tile width, fixed for the whole solve (0: look up)
};

Job make_job(const fe_problem *p, Slot *s) {
    Job j;
    j.p = p;
    j.slot = s;
    j.lanczos = method_of(p) != kMethodTrfoe;  // the truncated expansion scales by Gershgorin
    if (p->flags & FE_PTR_DEVICE) {
        j.H = p->Hp;
        j.ldh = p->ld;
    } else {
        j.H = s->Hcopy;
        j.ldh = p->n;
        j.stage = p->Hp;
        j.ldstage = p->ld;
    }
    return j;
}

template <typename T>
int ensure_pinned(fe_ctx *ctx, T **ptr, size_t *cap, size_t count) {
    if (count <= *cap) return FE_OK;
    if (*ptr) cudaFreeHost(*ptr);
    *ptr = nullptr;
    *cap = 0;
    const size_t c = std::max<size_t>(count, 4);
    FE_CUDA(ctx, cudaMallocHost(reinterpret_cast<void **>(ptr), sizeof(T) * c));
    *cap = c;
    return FE_OK;
}

int eng_init(fe_ctx *ctx, Engine &e, cudaStream_t user_stream) {
    if (user_stream) {
        e.stream = user_stream;
    } else {
        FE_CUDA(ctx, cudaStreamCreateWithFlags(&e.stream, cudaStreamNonBlocking));
        e.own_stream = true;
    }
    FE_CUDA(ctx, cudaMalloc(&e.d_err, sizeof(DevCtl)));
    {
        DevCtl c0{};
        c0.wait_ns = kWaitTimeoutNs;
        FE_CUDA(ctx, cudaMemcpy(e.d_err, &c0, sizeof(DevCtl), cudaMemcpyHostToDevice));
    }
    FE_CUDA(ctx, cudaMalloc(&e.d_flags, sizeof(StepFlags)));
    FE_CUDA(ctx, cudaMemset(e.d_flags, 0, sizeof(StepFlags)));
    FE_CUDA(ctx, cudaMalloc(&e.d_skws, sizeof(float) * kSkSlotFloats * ctx->num_sms));
    FE_CUDA(ctx, cudaMalloc(&e.d_skcnt, sizeof(int) * 2 * ctx->num_sms));
    FE_CUDA(ctx, cudaMemset(e.d_skcnt, 0, sizeof(int) * 2 * ctx->num_sms));
    FE_CUDA(ctx, cudaEventCreate(&e.ev0));
    FE_CUDA(ctx, cudaEventCreate(&e.ev1));
    FE_CUDA(ctx, cudaEventCreate(&e.ev_setup));
    FE_CUDA(ctx, cudaEventCreate(&e.ev_loop));
    return FE_OK;
}

void eng_free(Engine &e) {
    if (e.stream) cudaStreamSynchronize(e.stream);
    if (e.gexec) cudaGraphExecDestroy(e.gexec);
    if (e.graph) cudaGraphDestroy(e.graph);
    if (e.d_flags) cudaFree(e.d_flags);
    if (e.d_skws) cudaFree(e.d_skws);
    if (e.d_skcnt) cudaFree(e.d_skcnt);
    if (e.d_err) cudaFree(e.d_err);
    if (e.d_probs) cudaFree(e.d_probs);
    if (e.d_tiles) cudaFree(e.d_tiles);
    if (e.d_tiles64) cudaFree(e.d_tiles64);
    if (e.d_tilesD) cudaFree(e.d_tilesD);
    if (e.d_chk) cudaFree(e.d_chk);
    if (e.h_states) cudaFreeHost(e.h_states);
    if (e.h_done) cudaFreeHost(e.h_done);
    if (e.ev0) cudaEventDestroy(e.ev0);
    if (e.ev1) cudaEventDestroy(e.ev1);
    if (e.ev_setup) cudaEventDestroy(e.ev_setup);
    if (e.ev_loop) cudaEventDestroy(e.ev_loop);
    if (e.own_stream && e.stream) cudaStreamDestroy(e.stream);
    e = Engine();
}

int eng_upload(fe_ctx *ctx, Engine &e, const std::vector<Job> &jobs) {
    const int np = static_cast<int>(jobs.size());
    std::vector<MmaProb> hprobs(np);
    std::vector<TileEnt> tiles;
    std::vector<Tile64> tiles64;
    std::vector<TileEnt> tilesD;
    e.any_tc = e.any_fp64 = e.any_digit = false;
    e.off64.assign(np, 0);
    e.cnt64.assign(np, 0);
    for (int k = 0; k < np; ++k) {
        const Job &j = jobs[k];
        hprobs[k] = j.slot->hp;
        hprobs[k].H = j.H;
        hprobs[k].ldh = j.ldh;
        const bool fermi = method_of(j.p) == kMethodFermi;
        const bool trfoe = method_of(j.p) == kMethodTrfoe;  // its FP64 schedule runs digit products
        const uint32_t pr = prec_of(ctx, j.p);
        hprobs[k].tc_tile0 = static_cast<int>(tiles.size());
        hprobs[k].tc_ntiles = 0;
        if (pr != FE_PREC_FP64 || fermi) {
            e.any_tc = true;
            // a problem keeps its width for the whole solve: the control step
            // reduces the partial slots of the previous product's tiles
            const int bn = j.bn ? j.bn : tile_width(ctx, j.p->n, pr);
            const std::vector<TileEnt> &tl = (bn == kTileM) ? j.slot->tilesN : j.slot->tiles;
            for (TileEnt t : tl) { t.prob = k; tiles.push_back(t); }
            hprobs[k].tc_ntiles = static_cast<int>(tl.size());
            hprobs[k].ntiles = static_cast<int>(tl.size());
            hprobs[k].bn = bn;
        }
        e.off64[k] = static_cast<int>(tiles64.size());
        e.cnt64[k] = 0;
        if (pr == FE_PREC_FP64 && !fermi && !trfoe) {
            e.any_fp64 = true;
            for (Tile64 t : j.slot->tiles64) { t.prob = k; tiles64.push_back(t); }
            e.cnt64[k] = static_cast<int>(j.slot->tiles64.size());
        }
        if ((pr == FE_PREC_MIXED || pr == FE_PREC_TRY_FP16 || (trfoe && pr == FE_PREC_FP64)) && !fermi) {
            e.any_digit = true;
            for (TileEnt t : j.slot->tilesD) { t.prob = k; tilesD.push_back(t); }
        }
    }
    int rc = ensure_dev(ctx, &e.d_probs, &e.probs_cap, np);
    if (rc == FE_OK) rc = ensure_dev(ctx, &e.d_tiles, &e.tiles_cap, tiles.size());
    if (rc == FE_OK) rc = ensure_dev(ctx, &e.d_tiles64, &e.tiles64_cap, tiles64.size());
    if (rc == FE_OK) rc = ensure_dev(ctx, &e.d_tilesD, &e.tilesD_cap, tilesD.size());
    if (rc == FE_OK) rc = ensure_pinned(ctx, &e.h_states, &e.h_states_cap, np);
    if (rc == FE_OK) rc = ensure_pinned(ctx, &e.h_done, &e.h_done_cap, np + 1);  // + error word
    if (rc != FE_OK) return rc;
    FE_CUDA(ctx, cudaMemcpyAsync(e.d_probs, hprobs.data(), sizeof(MmaProb) * np,
                                 cudaMemcpyHostToDevice, e.stream));
    if (!tiles.empty())
        FE_CUDA(ctx, cudaMemcpyAsync(e.d_tiles, tiles.data(), sizeof(TileEnt) * tiles.size(),
                                     cudaMemcpyHostToDevice, e.stream));
    if (!tiles64.empty())
        FE_CUDA(ctx, cudaMemcpyAsync(e.d_tiles64, tiles64.data(), sizeof(Tile64) * tiles64.size(),
                                     cudaMemcpyHostToDevice, e.stream));
    if (!tilesD.empty())
        FE_CUDA(ctx, cudaMemcpyAsync(e.d_tilesD, tilesD.data(), sizeof(TileEnt) * tilesD.size(),
                                     cudaMemcpyHostToDevice, e.stream));
    // the copies read host vectors that go out of scope here
    FE_CUDA(ctx, cudaStreamSynchronize(e.stream));
    e.ntc = static_cast<int>(tiles.size());
    e.n64 = static_cast<int>(tiles64.size());
    e.nD = static_cast<int>(tilesD.size());
    return FE_OK;
}

// Set-up of the problems at table positions [k0, k1): Hp staging, initial
// state, bounds, X0 and the first control step.
int eng_setup(fe_ctx *ctx, Engine &e, const std::vector<Job> &jobs, int k0, int k1) {
    if (k1 <= k0) return FE_OK;
    cudaStream_t s = e.stream;
    const int m = k1 - k0;
    std::vector<int> tc_chk, f64_chk;  // problems certifying with the split-FP16 / FP64 kernel
    for (int k = k0; k < k1; ++k) {
        const Job &j = jobs[k];
        const int n = static_cast<int>(j.p->n);
        if (j.stage)
            FE_CUDA(ctx, cudaMemcpy2DAsync(j.slot->Hcopy, sizeof(double) * n, j.stage,
                                           sizeof(double) * j.ldstage, sizeof(double) * n, n,
                                           cudaMemcpyHostToDevice, s));
        init_state(ctx, j.p, &e.h_states[k]);
        e.h_states[k].lz_on = j.lanczos ? 1 : 0;
        if (!j.accel) e.h_states[k].acc_on = 0;
        FE_CUDA(ctx, cudaMemcpyAsync(j.slot->st, &e.h_states[k], sizeof(SolveState),
                                     cudaMemcpyHostToDevice, s));
        FE_CUDA(ctx, cudaMemsetAsync(j.slot->bad, 0, sizeof(int), s));
        k_bounds_rows<<<ceil_div(n, 8), 256, 0, s>>>(e.d_probs, k, j.slot->rowinfo, j.slot->bad);
        k_bounds_reduce<<<1, 1024, 0, s>>>(e.d_probs, k, j.slot->rowinfo, j.slot->bad);
        ctx->launches += 2;
        if (j.lanczos) (e.cnt64[k] > 0 ? f64_chk : tc_chk).push_back(k);
    }
    const bool any_lz = !tc_chk.empty() || !f64_chk.empty();
    if (any_lz) {
        // the estimate of every problem that takes one, all at once in one
        // cooperative launch (the kernel skips problems without lz_on)
        int vmax = 0;
        for (int k : tc_chk) vmax = std::max(vmax, static_cast<int>(jobs[k].p->n));
        for (int k : f64_chk) vmax = std::max(vmax, static_cast<int>(jobs[k].p->n));
        int vcap = std::min(vmax, kLzVcap);
        double narrow = ctx->lz_narrow.load(std::memory_order_relaxed);
        const MmaProb *probs = e.d_probs;
        DevCtl *ctl = e.d_err;
        unsigned *bar = &e.d_err->lz_bar;
        int kk0 = k0, mm = m;
        void *args[] = {&probs, &kk0, &mm, &vcap, &narrow, &ctl, &bar};
        FE_CUDA(ctx, cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
        FE_CUDA(ctx, cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_lanczos_run), dim3(ctx->lz_grid),
                                                 dim3(kLzThreads), args, sizeof(float) * vcap, s));
        ctx->launches += 1;
    }
    for (int k = k0; k < k1; ++k) k_init_x0<<<kInitBlocks, 256, 0, s>>>(e.d_probs, k);
    ctx->launches += m;
    if (any_lz) {
        // certify the estimates: kCheckSteps products over a table of just
        // those problems (the split-FP16 kernel takes them all in one launch,
        // the FP64 kernel one problem at a time), then X0 again on the
        // certified bounds
        if (!tc_chk.empty()) {
            const int nt = static_cast<int>(tc_chk.size());
            const MmaProb *tab = e.d_probs + tc_chk[0];
            if (tc_chk.back() - tc_chk[0] + 1 != nt) {  // not contiguous: gather the entries
                int rc = ensure_dev(ctx, &e.d_chk, &e.chk_cap, static_cast<size_t>(nt));
                if (rc != FE_OK) return rc;
                for (int q = 0; q < nt; ++q)
                    FE_CUDA(ctx, cudaMemcpyAsync(e.d_chk + q, e.d_probs + tc_chk[q], sizeof(MmaProb),
                                                 cudaMemcpyDeviceToDevice, s));
                tab = e.d_chk;
            }
            k_control<<<nt, 256, 0, s>>>(tab, nt, e.d_err, nullptr, 0, 0, 0, 0, 0u);
            for (int c = 0; c < kCheckSteps; ++c) {
                k_sym_mma<<<ctx->num_sms, kSymThreads, mma_smem_bytes(), s>>>(tab, nt, e.d_tiles, e.ntc, e.d_err,
                                                                           e.d_skws, e.d_skcnt);
                k_control<<<nt, 256, 0, s>>>(tab, nt, e.d_err, nullptr, 0, 0, 0, 0, 0u);
            }
            ctx->launches += 1 + 2 * kCheckSteps;
        }
        for (int k : f64_chk) {
            const MmaProb *one = e.d_probs + k;
            k_control<<<1, 256, 0, s>>>(one, 1, e.d_err, nullptr, 0, 0, 0, 0, 0u);
            for (int c = 0; c < kCheckSteps; ++c) {
                k_fp64_step<<<std::max(1, std::min(e.cnt64[k], 4 * ctx->num_sms)), 256, 0, s>>>(
                    e.d_probs, e.d_tiles64 + e.off64[k], e.cnt64[k]);
                k_control<<<1, 256, 0, s>>>(one, 1, e.d_err, nullptr, 0, 0, 0, 0, 0u);
            }
            ctx->launches += 1 + 2 * kCheckSteps;
        }
        k_check_bounds<<<m, 32, 0, s>>>(e.d_probs, k0);
        ++ctx->launches;
        for (int k : tc_chk) k_init_x0<<<kInitBlocks, 256, 0, s>>>(e.d_probs, k);
        for (int k : f64_chk) k_init_x0<<<kInitBlocks, 256, 0, s>>>(e.d_probs, k);
        ctx->launches += static_cast<long long>(tc_chk.size() + f64_chk.size());
    }
    k_control<<<m, 256, 0, s>>>(e.d_probs + k0, m, e.d_err, nullptr, 0, 0, 0, 0, 0u);
    ++ctx->launches;
    // the state images must stay valid until their copies ran
    FE_CUDA(ctx, cudaStreamSynchronize(s));
    return FE_OK;
}

// `count` expansion steps over every problem in the table; with `pev` each
// tensor-core and FP64 launch is bracketed by events (4 per step).
void eng_steps(fe_ctx *ctx, Engine &e, int np, int count, const std::vector<cudaEvent_t> *pev) {
    cudaStream_t s = e.stream;
    const int grid_tc = ctx->num_sms;  // the kernel itself uses at most (work / largest tile) CTAs
    const int grid_64 = std::max(1, std::min(e.n64, 4 * ctx->num_sms));
    const size_t smem = mma_smem_bytes();
    const int grid_d = std::max(1, std::min(e.nD, ctx->num_sms));
    for (int it = 0; it < count; ++it) {
        if (pev) cudaEventRecord((*pev)[4 * it + 0], s);
        if (e.any_tc) {
            k_sym_mma<<<grid_tc, kSymThreads, smem, s>>>(e.d_probs, np, e.d_tiles, e.ntc, e.d_err, e.d_skws,
                                                          e.d_skcnt);
            ++ctx->launches;
        }
        if (pev) cudaEventRecord((*pev)[4 * it + 1], s);
        if (pev) cudaEventRecord((*pev)[4 * it + 2], s);
        if (e.any_fp64) {
            k_fp64_step<<<grid_64, 256, 0, s>>>(e.d_probs, e.d_tiles64, e.n64);
            ++ctx->launches;
        }
        if (e.any_digit) {
            k_digit_prep<<<2 * ctx->num_sms, 256, 0, s>>>(e.d_probs, np);
            k_digit_mma<<<grid_d, kMmaThreads, digit_smem_bytes(), s>>>(e.d_probs, e.d_tilesD, e.nD,
                                                                        e.d_err);
            ctx->launches += 2;
        }
        if (pev) cudaEventRecord((*pev)[4 * it + 3], s);
        k_control<<<np, 256, 0, s>>>(e.d_probs, np, e.d_err, nullptr, 0, 0, 0, 0, 0u);
        ++ctx->launches;
    }
}

// Output kernels of the problem at table position k and the read-back of its
// state into e.h_states[k] (asynchronous).
int eng_finish(fe_ctx *ctx, Engine &e, int k, const Job &j) {
    cudaStream_t s = e.stream;
    const fe_problem *p = j.p;
    double *dout = nullptr;
    long long ldd = p->n;
    bool staged = false;
    if (p->D) {
        if (p->flags & FE_PTR_DEVICE) {
            dout = p->D;
            ldd = p->ld;
        } else {
            // page-locked host memory that the device can address: the output
            // kernel writes D there directly (one pass over the host link, no
            // staging buffer or separate copy); other host memory is staged
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, p->D) == cudaSuccess && a.type == cudaMemoryTypeHost &&
                a.devicePointer != nullptr) {
                dout = static_cast<double *>(a.devicePointer);
                ldd = p->ld;
            } else {
                cudaGetLastError();  // a pointer CUDA does not know is not an error here
                dout = j.slot->Dtmp;
                staged = true;
            }
        }
    }
    k_finalize<<<kFinBlocks, 256, 0, s>>>(e.d_probs, k, dout, ldd);
    k_finalize_reduce<<<1, 512, 0, s>>>(e.d_probs, k);
    ctx->launches += 2;
    if (staged)
        FE_CUDA(ctx, cudaMemcpy2DAsync(p->D, sizeof(double) * p->ld, j.slot->Dtmp,
                                       sizeof(double) * p->n, sizeof(double) * p->n, p->n,
                                       cudaMemcpyDeviceToHost, s));
    FE_CUDA(ctx, cudaMemcpyAsync(&e.h_states[k], j.slot->st, sizeof(SolveState),
                                 cudaMemcpyDeviceToHost, s));
    return FE_OK;
}

void fill_result(const SolveState &st, int herr, double ms, fe_result &r) {
    memset(&r, 0, sizeof(r));
    r.status = st.status == 0 ? FE_OK : st.status;
    if (herr != 0) r.status = FE_ETIMEOUT;
    r.iters = st.iter;
    for (int q = 0; q < 3; ++q) r.iters_by_phase[q] = st.it_phase[q];
    if (st.method == kMethodFermi) r.iters_by_phase[3] = st.ft_stage;
    r.e_band = st.e_band;
    r.trace = st.trace;
    r.idem_fro = st.idem_fro;
    r.mu = st.mu;
    r.eps_min = st.emin;
    r.eps_max = st.emax;
    r.ms = ms;
}

// The step loop of the uploaded table as an instantiated CUDA graph (built
// once per table layout): the control kernel sets the loop condition and the
// kernel switches of the next step on the device, so exactly the steps and
// kernels that have work run, with no host round trip.
int eng_graph(fe_ctx *ctx, Engine &e, int np) {
    std::vector<uintptr_t> key = {reinterpret_cast<uintptr_t>(e.d_probs), reinterpret_cast<uintptr_t>(e.d_tiles),
                                  reinterpret_cast<uintptr_t>(e.d_tiles64), reinterpret_cast<uintptr_t>(e.d_tilesD),
                                  static_cast<uintptr_t>(np), static_cast<uintptr_t>(e.ntc),
                                  static_cast<uintptr_t>(e.n64), static_cast<uintptr_t>(e.nD),
                                  static_cast<uintptr_t>(e.any_tc), static_cast<uintptr_t>(e.any_fp64),
                                  static_cast<uintptr_t>(e.any_digit)};
    if (e.gexec && key == e.gkey) return FE_OK;
    if (e.gexec) cudaGraphExecDestroy(e.gexec);
    if (e.graph) cudaGraphDestroy(e.graph);
    e.gexec = nullptr;
    e.graph = nullptr;
    e.gkey.clear();
    cudaGraph_t g;
    FE_CUDA(ctx, cudaGraphCreate(&g, 0));
    e.graph = g;
    cudaGraphConditionalHandle hl = 0, ht = 0, hf = 0, hd = 0;
    // defaults: the first step runs every kernel family (each skips problems
    // whose step is not its own); later steps follow the control kernel.
    // A handle exists only for a family the graph contains.
    unsigned hvalid = kStepActive;
    FE_CUDA(ctx, cudaGraphConditionalHandleCreate(&hl, g, 1, cudaGraphCondAssignDefault));
    if (e.any_tc) {
        FE_CUDA(ctx, cudaGraphConditionalHandleCreate(&ht, g, 1, cudaGraphCondAssignDefault));
        hvalid |= kStepTc;
    }
    if (e.any_fp64) {
        FE_CUDA(ctx, cudaGraphConditionalHandleCreate(&hf, g, 1, cudaGraphCondAssignDefault));
        hvalid |= kStepFp64;
    }
    if (e.any_digit) {
        FE_CUDA(ctx, cudaGraphConditionalHandleCreate(&hd, g, 1, cudaGraphCondAssignDefault));
        hvalid |= kStepDigit;
    }
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hl;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn;
    FE_CUDA(ctx, cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaGraphNode_t prev = nullptr;
    // an IF node in the loop body after `prev`; returns its body graph
    auto add_if = [&](cudaGraphConditionalHandle h, cudaGraph_t *ib) -> cudaError_t {
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t in;
        cudaError_t r = cudaGraphAddNode(&in, body, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &ip);
        if (r == cudaSuccess) {
            prev = in;
            *ib = ip.conditional.phGraph_out[0];
        }
        return r;
    };
    auto add_kernel = [&](cudaGraph_t gr, const void *fn, int grid, int block, size_t smem, void **args,
                          cudaGraphNode_t *dep, cudaGraphNode_t *out) -> cudaError_t {
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void *>(fn);
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.sharedMemBytes = static_cast<unsigned>(smem);
        kp.kernelParams = args;
        return cudaGraphAddKernelNode(out, gr, dep, dep ? 1 : 0, &kp);
    };
    const MmaProb *probs = e.d_probs;
    DevCtl *err = e.d_err;
    cudaGraphNode_t kn, kn2;
    if (e.any_tc) {
        cudaGraph_t ib;
        FE_CUDA(ctx, add_if(ht, &ib));
        const TileEnt *tl = e.d_tiles;
        int nt = e.ntc, npp = np;
        float *skws = e.d_skws;
        int *skcnt = e.d_skcnt;
        void *args[] = {&probs, &npp, &tl, &nt, &err, &skws, &skcnt};
        FE_CUDA(ctx, add_kernel(ib, reinterpret_cast<const void *>(k_sym_mma), ctx->num_sms, kSymThreads,
                                mma_smem_bytes(), args, nullptr, &kn));
    }
    if (e.any_fp64) {
        cudaGraph_t ib;
        FE_CUDA(ctx, add_if(hf, &ib));
        const Tile64 *tl = e.d_tiles64;
        int nt = e.n64;
        void *args[] = {&probs, &tl, &nt};
        FE_CUDA(ctx, add_kernel(ib, reinterpret_cast<const void *>(k_fp64_step),
                                std::max(1, std::min(e.n64, 4 * ctx->num_sms)), 256, 0, args, nullptr, &kn));
    }
    if (e.any_digit) {
        cudaGraph_t ib;
        FE_CUDA(ctx, add_if(hd, &ib));
        int npp = np;
        void *pargs[] = {&probs, &npp};
        FE_CUDA(ctx, add_kernel(ib, reinterpret_cast<const void *>(k_digit_prep), 2 * ctx->num_sms, 256, 0,
                                pargs, nullptr, &kn));
        const TileEnt *tl = e.d_tilesD;
        int nt = e.nD;
        void *args[] = {&probs, &tl, &nt, &err};
        FE_CUDA(ctx, add_kernel(ib, reinterpret_cast<const void *>(k_digit_mma),
                                std::max(1, std::min(e.nD, ctx->num_sms)), kMmaThreads, digit_smem_bytes(),
                                args, &kn, &kn2));
    }
    {
        int npp = np;
        StepFlags *fl = e.d_flags;
        void *args[] = {&probs, &npp, &err, &fl, &hl, &ht, &hf, &hd, &hvalid};
        FE_CUDA(ctx, add_kernel(body, reinterpret_cast<const void *>(k_control), np, 256, 0, args,
                                prev ? &prev : nullptr, &kn));
    }
    FE_CUDA(ctx, cudaGraphInstantiate(&e.gexec, g, 0));
    e.gkey = key;
    return FE_OK;
}

// Run validated problems on acquired slots to completion (blocking calls).
int run_problems_once(fe_ctx *ctx, const std::vector<Job> &jobs, fe_result *rs) {
    Engine &e = ctx->eng;
    const int np = static_cast<int>(jobs.size());
    cudaStream_t s = e.stream;
    int rc = eng_upload(ctx, e, jobs);
    if (rc != FE_OK) return rc;
    FE_CUDA(ctx, cudaMemsetAsync(e.d_err, 0, sizeof(int), s));
    FE_CUDA(ctx, cudaMemsetAsync(e.d_skcnt, 0, sizeof(int) * 2 * ctx->num_sms, s));
    FE_CUDA(ctx, cudaEventRecord(e.ev0, s));
    rc = eng_setup(ctx, e, jobs, 0, np);
    if (rc != FE_OK) return rc;
    FE_CUDA(ctx, cudaEventRecord(e.ev_setup, s));
    int total_iters = 0;
    for (int k = 0; k < np; ++k) total_iters = std::max(total_iters, e.h_states[k].max_iters);
    // one step = product + control; +8 covers the phase hand-offs
    const int nloop = total_iters + 8;
    if (ctx->prof) {
        while (ctx->pev.size() < static_cast<size_t>(4 * nloop)) {
            cudaEvent_t ev;
            FE_CUDA(ctx, cudaEventCreate(&ev));
            ctx->pev.push_back(ev);
        }
    }
    const bool use_graph = !ctx->prof;  // per-launch events need plain launches
    if (use_graph) {
        rc = eng_graph(ctx, e, np);
        if (rc != FE_OK) return rc;
        FE_CUDA(ctx, cudaMemsetAsync(e.d_flags, 0, sizeof(StepFlags), s));
        FE_CUDA(ctx, cudaGraphLaunch(e.gexec, s));
        FE_CUDA(ctx, cudaMemcpyAsync(&e.h_flags, e.d_flags, sizeof(StepFlags), cudaMemcpyDeviceToHost, s));
    } else {
        eng_steps(ctx, e, np, nloop, ctx->prof ? &ctx->pev : nullptr);
    }
    FE_CUDA(ctx, cudaEventRecord(e.ev_loop, s));
    for (int k = 0; k < np; ++k) {
        rc = eng_finish(ctx, e, k, jobs[k]);
        if (rc != FE_OK) return rc;
    }
    FE_CUDA(ctx, cudaEventRecord(e.ev1, s));
    FE_CUDA(ctx, cudaGetLastError());
    int herr = 0;
    FE_CUDA(ctx, cudaMemcpyAsync(&herr, e.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    FE_CUDA(ctx, cudaStreamSynchronize(s));
    float ms = 0.0f, ms_setup = 0.0f, ms_loop = 0.0f, ms_fin = 0.0f;
    cudaEventElapsedTime(&ms, e.ev0, e.ev1);
    cudaEventElapsedTime(&ms_setup, e.ev0, e.ev_setup);
    cudaEventElapsedTime(&ms_loop, e.ev_setup, e.ev_loop);
    cudaEventElapsedTime(&ms_fin, e.ev_loop, e.ev1);
    ctx->phase_ms[0] = ms_setup;
    ctx->phase_ms[1] = ms_loop;
    ctx->phase_ms[2] = ms_fin;
    ctx->phase_ms[3] = use_graph ? static_cast<double>(e.h_flags.n_body) : static_cast<double>(nloop);
    if (use_graph) {
        // kernels the graph ran: a control per step, every family once in the
        // first step, then the families the control kernel switched on
        const StepFlags &fl = e.h_flags;
        ctx->launches += fl.n_body + (e.any_tc ? 1 : 0) + (e.any_fp64 ? 1 : 0) + (e.any_digit ? 2 : 0) +
                         fl.n_tc + fl.n_fp64 + 2ll * fl.n_digit;
    }
    if (ctx->prof) {
        // launches that did work: the phases run in order (single FP16, split,
        // FP64), so the first it_phase[0] + it_phase[1] tensor-core launches
        // and the it_phase[2] FP64 launches after them were active; a
        // finite-temperature solve uses the tensor cores for every step
        int tc_active = 0, fp_active = 0;
        for (int k = 0; k < np; ++k) {
            const SolveState &st = e.h_states[k];
            const int tc = (st.method == kMethodFermi) ? st.iter : st.it_phase[0] + st.it_phase[1];
            tc_active = std::max(tc_active, tc);
            fp_active = std::max(fp_active, st.method == kMethodFermi ? 0 : st.it_phase[2]);
        }
        double tc_ms = 0, fp_ms = 0, tc_all = 0;
        ctx->prof_steps.assign(nloop, 0.0);
        for (int it = 0; it < nloop; ++it) {
            float a = 0, b = 0;
            cudaEventElapsedTime(&a, ctx->pev[4 * it + 0], ctx->pev[4 * it + 1]);
            cudaEventElapsedTime(&b, ctx->pev[4 * it + 2], ctx->pev[4 * it + 3]);
            ctx->prof_steps[it] = a;
            tc_all += a;
            if (it < tc_active) tc_ms += a;
            if (it >= tc_active && it < tc_active + fp_active) fp_ms += b;
        }
        ctx->prof_out[0] = tc_ms;
        ctx->prof_out[1] = tc_active;
        ctx->prof_out[2] = fp_ms;
        ctx->prof_out[3] = fp_active;
        ctx->prof_out[4] = ms;
        ctx->prof_out[5] = static_cast<double>(ctx->launches.load());
        ctx->prof_out[6] = tc_all;
        ctx->prof_out[7] = e.any_tc ? nloop : 0;
        // by kind of step: the k-th pass of the loop runs the k-th step issued
        for (int q = 0; q < 8; ++q) {
            ctx->prof_kind_ms[q] = 0.0;
            ctx->prof_kind_n[q] = 0;
        }
        const SolveState &s0 = e.h_states[0];
        for (int it = 0; it < nloop && it < s0.nctl && it < kKindLog; ++it) {
            const int kd = s0.kind_log[it];
            if (kd <= kNone || kd > 7) continue;
            float a = 0;
            const bool tc = (kd == kTcSingle || kd == kTcSplit || kd == kTcElem || kd == kTcDelta);
            cudaEventElapsedTime(&a, ctx->pev[4 * it + (tc ? 0 : 2)], ctx->pev[4 * it + (tc ? 1 : 3)]);
            ctx->prof_kind_ms[kd] += a;
            ctx->prof_kind_n[kd] += 1;
        }
    }
    int first_bad = FE_OK;
    for (int k = 0; k < np; ++k) {
        fill_result(e.h_states[k], herr, ms, rs[k]);
        if (rs[k].status != FE_OK && first_bad == FE_OK) first_bad = rs[k].status;
    }
    if (herr != 0) set_err(ctx, FE_ETIMEOUT, "device wait timed out (code " + std::to_string(herr) + ")");
    else if (first_bad == FE_EINVAL) set_err(ctx, FE_EINVAL, "NaN or Inf in Hp");
    else if (first_bad == FE_ENOTCONV) set_err(ctx, FE_ENOTCONV, "iteration cap reached");
    return first_bad;
}

// As run_problems_once; a problem whose spectral-bound estimate proved too
// tight (an eigenvalue of X left [0, 1]) is solved again from the Gershgorin
// bounds, which always contain the spectrum, and an FE_METHOD_ASP2 problem
// whose HOMO/LUMO estimates proved inconsistent with its spectrum is solved
// again as plain SP2 (at most one of each, in that order of discovery);
// fe_result.iters then includes the products of the abandoned attempts.
int run_problems(fe_ctx *ctx, const std::vector<Job> &jobs, fe_result *rs) {
    int rc = run_problems_once(ctx, jobs, rs);
    std::vector<Job> cur = jobs;
    std::vector<int> where(jobs.size());
    for (size_t k = 0; k < jobs.size(); ++k) where[k] = static_cast<int>(k);
    std::vector<int> wasted(jobs.size(), 0);
    for (int round = 0; round < 2; ++round) {
        std::vector<Job> again;
        std::vector<int> at;
        for (size_t q = 0; q < cur.size(); ++q) {
            const int k = where[q];
            const int st = rs[k].status;
            if (st == kStatusEscaped && cur[q].lanczos) {
                Job j = cur[q];
                j.lanczos = false;
                again.push_back(j);
                at.push_back(k);
            } else if (st == kStatusAccelFailed && cur[q].accel) {
                Job j = cur[q];
                j.accel = false;
                again.push_back(j);
                at.push_back(k);
            }
        }
        if (again.empty()) break;
        std::vector<fe_result> rr(again.size());
        run_problems_once(ctx, again, rr.data());
        for (size_t q = 0; q < again.size(); ++q) {
            wasted[at[q]] += rs[at[q]].iters;
            rs[at[q]] = rr[q];
        }
        cur.swap(again);
        where.swap(at);
    }
    rc = FE_OK;
    for (size_t k = 0; k < jobs.size(); ++k) {
        if (rs[k].status == kStatusEscaped || rs[k].status == kStatusAccelFailed) rs[k].status = FE_ENOTCONV;
        rs[k].iters += wasted[k];
        if (rs[k].status != FE_OK && rc == FE_OK) rc = rs[k].status;
    }
    return rc;
}

// ---------------------------------------------------------------- serving
// Continuous batching behind fe_submit / fe_poll.  One worker thread owns a
// second engine (its own stream).  Each tick it starts the waiting requests
// that fit the free part of the HBM budget (first fit, in submission order),
// runs kServeSteps expansion steps over every running request at once, reads
// the done flags, and finishes the requests that converged (D written, slot
// released, result published for fe_poll).  Requests therefore join and
// leave the batch at step granularity, and short solves are not held back by
// long ones.

constexpr int kServeSteps = 8;
constexpr size_t kMaxTickets = 1 << 16;
constexpr double kAdmitWaitMs = 60000.0;

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Publish a final result; the worker does not touch r afterwards.
void publish(fe_ctx *ctx, Req *r, const fe_result &res) {
    std::lock_guard<std::mutex> lk(ctx->qmu);
    r->res = res;
    r->res.ms = ms_since(r->t_submit);
    r->done = true;
}

void fail_req(fe_ctx *ctx, Req *r, int status) {
    if (r->slot) release_slot(ctx, r->slot);
    r->slot = nullptr;
    fe_result res;
    memset(&res, 0, sizeof(res));
    res.status = status;
    publish(ctx, r, res);
}

Job job_of(Req *r) {
    Job j;
    j.p = &r->p;
    j.slot = r->slot;
    j.H = r->slot->Hcopy;
    j.ldh = r->p.n;
    if (!r->staged) {
        j.stage = r->hbuf.data();
        j.ldstage = r->p.n;
    }
    j.lanczos = !r->gershgorin && method_of(&r->p) != kMethodTrfoe;
    j.accel = !r->accel_off;
    j.bn = r->bn;
    return j;
}

void serve_loop(fe_ctx *ctx) {
    cudaSetDevice(ctx->device);
    Engine &e = ctx->seng;
    std::vector<Req *> running;
    for (;;) {
        std::vector<Req *> cand;
        {
            std::unique_lock<std::mutex> lk(ctx->qmu);
            ctx->qcv.wait(lk, [&] { return ctx->stop || !ctx->waiting.empty() || !running.empty(); });
            if (ctx->stop) break;
            cand.assign(ctx->waiting.begin(), ctx->waiting.end());
        }
        // admission, outside the queue lock (slot allocation may call cudaMalloc)
        std::vector<Req *> started, failed;
        for (Req *r : cand) {
            if (!r->slot) {
                Slot *s = nullptr;
                if (acquire_slot(ctx, static_cast<int>(r->p.n), slot_method(&r->p), &s) != FE_OK) {
                    if (!r->deferred) {
                        r->deferred = true;
                        std::lock_guard<std::mutex> lk(ctx->qmu);
                        ctx->n_deferred += 1;
                    }
                    // blocking solves may hold the memory for a while; with
                    // nothing of ours running, give up after kAdmitWaitMs
                    if (running.empty() && ms_since(r->t_submit) > kAdmitWaitMs) failed.push_back(r);
                    continue;
                }
                r->slot = s;
            }
            if (r->bn == 0) r->bn = tile_width(ctx, r->p.n, prec_of(ctx, &r->p));
            started.push_back(r);
        }
        if (!started.empty() || !failed.empty()) {
            std::lock_guard<std::mutex> lk(ctx->qmu);
            auto gone = [&](Req *r) {
                return std::find(started.begin(), started.end(), r) != started.end() ||
                       std::find(failed.begin(), failed.end(), r) != failed.end();
            };
            ctx->waiting.erase(std::remove_if(ctx->waiting.begin(), ctx->waiting.end(), gone),
                               ctx->waiting.end());
        }
        for (Req *r : failed) fail_req(ctx, r, FE_ENOMEM);
        {
            std::lock_guard<std::mutex> lk(ctx->qmu);
            ctx->peak_running = std::max<long long>(ctx->peak_running,
                                                    static_cast<long long>(running.size() + started.size()));
        }
        if (running.empty() && started.empty()) {
            // requests wait for memory held elsewhere: poll again shortly
            std::unique_lock<std::mutex> lk(ctx->qmu);
            ctx->qcv.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }

        const int k0 = static_cast<int>(running.size());
        std::vector<Req *> all = running;
        all.insert(all.end(), started.begin(), started.end());
        std::vector<Job> jobs;
        for (Req *r : all) jobs.push_back(job_of(r));
        const int np = static_cast<int>(all.size());
        int rc = FE_OK;
        cudaMemsetAsync(e.d_err, 0, sizeof(int), e.stream);
        cudaMemsetAsync(e.d_skcnt, 0, sizeof(int) * 2 * ctx->num_sms, e.stream);
        if (!started.empty()) {
            rc = eng_upload(ctx, e, jobs);
            if (rc == FE_OK) rc = eng_setup(ctx, e, jobs, k0, np);
        }
        int herr = 0;
        if (rc == FE_OK) {
            eng_steps(ctx, e, np, kServeSteps, nullptr);
            for (int k = 0; k < np; ++k)
                cudaMemcpyAsync(&e.h_done[k], &all[k]->slot->st->done, sizeof(int),
                                cudaMemcpyDeviceToHost, e.stream);
            cudaMemcpyAsync(&e.h_done[np], e.d_err, sizeof(int), cudaMemcpyDeviceToHost, e.stream);
            const cudaError_t ce = cudaStreamSynchronize(e.stream);
            if (ce != cudaSuccess) rc = cuda_fail(ctx, ce, "serving step");
            else herr = e.h_done[np];
        }
        if (rc != FE_OK || herr != 0) {
            for (Req *r : all) fail_req(ctx, r, rc != FE_OK ? rc : FE_ETIMEOUT);
            running.clear();
            continue;
        }
        // finish the converged ones
        std::vector<Req *> next;
        std::vector<int> fin;
        for (int k = 0; k < np; ++k) {
            if (e.h_done[k]) fin.push_back(k);
            else next.push_back(all[k]);
        }
        for (int k : fin) {
            rc = eng_finish(ctx, e, k, jobs[k]);
            if (rc != FE_OK) break;
        }
        if (rc == FE_OK && !fin.empty()) {
            const cudaError_t ce = cudaStreamSynchronize(e.stream);
            if (ce != cudaSuccess) rc = cuda_fail(ctx, ce, "serving finish");
        }
        std::vector<Req *> redo;
        for (int k : fin) {
            Req *r = all[k];
            fe_result res;
            fill_result(e.h_states[k], 0, 0.0, res);
            if (rc != FE_OK) res.status = rc;
            if ((res.status == kStatusEscaped && !r->gershgorin) ||
                (res.status == kStatusAccelFailed && !r->accel_off)) {
                // start again (Hp is in the slot): from the Gershgorin bounds,
                // or as plain SP2 when the HOMO/LUMO estimates were inconsistent
                if (res.status == kStatusEscaped) r->gershgorin = true;
                else r->accel_off = true;
                r->wasted += res.iters;
                r->staged = true;
                redo.push_back(r);
                continue;
            }
            if (res.status == kStatusEscaped || res.status == kStatusAccelFailed) res.status = FE_ENOTCONV;
            res.iters += r->wasted;
            release_slot(ctx, r->slot);
            r->slot = nullptr;
            publish(ctx, r, res);
        }
        if (!redo.empty()) {
            std::lock_guard<std::mutex> lk(ctx->qmu);
            for (Req *r : redo) ctx->waiting.push_front(r);
        }
        running.swap(next);
        if (!fin.empty() && !running.empty()) {
            // rebuild the table without the finished requests
            std::vector<Job> rest;
            for (Req *r : running) rest.push_back(job_of(r));
            if (eng_upload(ctx, e, rest) != FE_OK) {
                for (Req *r : running) fail_req(ctx, r, FE_ECUDA);
                running.clear();
            }
        }
    }
    // shutting down: let queued work drain from the stream; fe_destroy frees the rest
    cudaStreamSynchronize(e.stream);
    for (Req *r : running) release_slot(ctx, r->slot);
}

// ---------------------------------------------------------------- tile table file
// Text: a header line "fe-autotune 1", then one line per entry:
// <128-row panels> <FE_PREC_* value> <tile width> <ms with 256> <ms with 128>.

int load_tune(fe_ctx *ctx, const std::string &path) {
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return FE_OK;  // no table yet
    char head[32] = {};
    int ver = 0;
    int rc = FE_OK;
    if (fscanf(f, "%31s %d", head, &ver) != 2 || std::string(head) != "fe-autotune" || ver != 1) {
        rc = set_err(nullptr, FE_EINVAL, "autotune file " + path + ": bad header");
    } else {
        int T = 0, bn = 0;
        unsigned prec = 0;
        double a = 0, b = 0;
        int got;
        while ((got = fscanf(f, "%d %u %d %lf %lf", &T, &prec, &bn, &a, &b)) == 5) {
            if (T < 1 || (bn != kTileM && bn != kTileN) || (prec & ~FE_PREC_MASK) != 0) {
                rc = set_err(nullptr, FE_EINVAL, "autotune file " + path + ": bad entry");
                break;
            }
            ctx->tune[{T, prec}] = TuneEnt{bn, a, b};
        }
        if (rc == FE_OK && got != EOF) rc = set_err(nullptr, FE_EINVAL, "autotune file " + path + ": bad entry");
    }
    fclose(f);
    return rc;
}

// caller holds ctx->tmu
int save_tune(fe_ctx *ctx) {
    if (ctx->tune_path.empty()) return FE_OK;
    FILE *f = fopen(ctx->tune_path.c_str(), "w");
    if (!f) return set_err(ctx, FE_EINVAL, "cannot write autotune file " + ctx->tune_path);
    fprintf(f, "fe-autotune 1\n");
    for (const auto &kv : ctx->tune)
        fprintf(f, "%d %u %d %.6f %.6f\n", kv.first.first, kv.first.second, kv.second.bn, kv.second.ms_w,
                kv.second.ms_n);
    const bool ok = fclose(f) == 0;
    return ok ? FE_OK : set_err(ctx, FE_EINVAL, "cannot write autotune file " + ctx->tune_path);
}

}  // namespace

// ============================================================== C ABI

extern "C" int fe_create(fe_ctx **out, const fe_config *cfg) {
    if (!out) return set_err(nullptr, FE_EINVAL, "out is NULL");
    *out = nullptr;
    fe_config c{};
    if (cfg) c = *cfg;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return set_err(nullptr, FE_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    if (c.device < 0 || c.device >= ndev) return set_err(nullptr, FE_EINVAL, "bad device ordinal");
    if ((e = cudaSetDevice(c.device)) != cudaSuccess)
        return set_err(nullptr, FE_ECUDA, cudaGetErrorString(e));
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, c.device);
    if (prop.major != 10 || prop.minor != 3)
        return set_err(nullptr, FE_ECUDA, "this library is built for sm_103a (GB300) only");
    if (!get_encode()) return set_err(nullptr, FE_ECUDA, "cuTensorMapEncodeTiled not available");
    fe_ctx *ctx = new fe_ctx();
    if (c.autotune_path) {
        ctx->tune_path = c.autotune_path;
        const int lrc = load_tune(ctx, ctx->tune_path);
        if (lrc != FE_OK) {
            const std::string why = g_err;
            delete ctx;
            return set_err(nullptr, lrc, why);
        }
    }
    ctx->device = c.device;
    ctx->num_sms = prop.multiProcessorCount;
    ctx->max_iters = c.max_iters > 0 ? c.max_iters : 100;
    ctx->prec_default = c.precision_policy;
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    ctx->budget = c.hbm_budget_bytes ? c.hbm_budget_bytes : static_cast<size_t>(0.8 * freeb);
    int rc = eng_init(ctx, ctx->eng, static_cast<cudaStream_t>(c.cuda_stream));
    if (rc == FE_OK) rc = eng_init(ctx, ctx->seng, nullptr);
    if (rc == FE_OK && cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = set_err(nullptr, FE_ECUDA, "copy stream");
    if (rc == FE_OK && (cudaFuncSetAttribute(k_sym_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(mma_smem_bytes())) != cudaSuccess ||
                        cudaFuncSetAttribute(k_digit_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(digit_smem_bytes())) != cudaSuccess ||
                        cudaFuncSetAttribute(k_gemm_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(gemm_smem_bytes())) != cudaSuccess ||
                        cudaFuncSetAttribute(k_lanczos_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(sizeof(float) * kLzVcap)) != cudaSuccess))
        rc = set_err(nullptr, FE_ECUDA, std::string("context setup: ") + cudaGetErrorString(cudaGetLastError()));
    if (rc == FE_OK) {
        // the Lanczos launch waits at grid barriers, so all its blocks must be
        // resident at once: a cooperative launch no larger than the occupancy
        // allows with the largest staged vector
        int coop = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c.device) != cudaSuccess || !coop ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lanczos_run, kLzThreads,
                                                          sizeof(float) * kLzVcap) != cudaSuccess ||
            per_sm < 1)
            rc = set_err(nullptr, FE_ECUDA, "cooperative launch of k_lanczos_run unavailable");
        else
            ctx->lz_grid = std::min(kLzBlocks, per_sm * ctx->num_sms);
    }
    if (rc == FE_OK) {
        // the register hand-off inside the split-FP16 kernel assumes this allocation
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_sym_mma) != cudaSuccess || fa.numRegs != kSymLaunchRegs)
            rc = set_err(nullptr, FE_ECUDA, "k_sym_mma was compiled with " + std::to_string(fa.numRegs) +
                                                " registers per thread; the kernel needs " +
                                                std::to_string(kSymLaunchRegs));
    }
    if (rc != FE_OK) {
        const std::string why = g_err;
        fe_destroy(ctx);
        return set_err(nullptr, rc, why);
    }
    *out = ctx;
    return FE_OK;
}

extern "C" int fe_destroy(fe_ctx *ctx) {
    if (!ctx) return FE_OK;
    {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        ctx->stop = true;
    }
    ctx->qcv.notify_all();
    if (ctx->worker.joinable()) ctx->worker.join();
    cudaSetDevice(ctx->device);
    eng_free(ctx->eng);
    eng_free(ctx->seng);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (auto &kv : ctx->reqs) delete kv.second;
    ctx->reqs.clear();
    for (Slot *s : ctx->slots) {
        if (s->arena) cudaFree(s->arena);
        delete s;
    }
    ctx->slots.clear();
    for (cudaEvent_t ev : ctx->pev) cudaEventDestroy(ev);
    if (ctx->gws) cudaFree(ctx->gws);
    if (ctx->d_gargs) cudaFree(ctx->d_gargs);
    if (ctx->d_gtiles) cudaFree(ctx->d_gtiles);
    if (ctx->d_amax) cudaFree(ctx->d_amax);
    delete ctx;
    return FE_OK;
}

extern "C" int fe_solve(fe_ctx *ctx, const fe_problem *p, fe_result *r) {
    if (!ctx) return set_err(nullptr, FE_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    fe_result dummy;
    if (!r) r = &dummy;
    memset(r, 0, sizeof(*r));
    int rc = validate(ctx, p);
    if (rc != FE_OK) return r->status = rc;
    cudaSetDevice(ctx->device);
    Slot *s = nullptr;
    rc = acquire_slot(ctx, static_cast<int>(p->n), slot_method(p), &s);
    if (rc != FE_OK) return r->status = rc;
    std::vector<Job> jobs{make_job(p, s)};
    rc = run_problems(ctx, jobs, r);
    release_slot(ctx, s);
    if (r->status == FE_OK && rc != FE_OK) r->status = rc;
    return rc;
}

extern "C" int fe_solve_batch(fe_ctx *ctx, int count, const fe_problem *ps, fe_result *rs) {
    if (!ctx) return set_err(nullptr, FE_EINVAL, "ctx is NULL");
    if (count < 0 || (count > 0 && (!ps || !rs))) return set_err(ctx, FE_EINVAL, "bad batch arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (count == 0) return FE_OK;
    cudaSetDevice(ctx->device);
    std::vector<Job> jobs;
    std::vector<int> idx;
    int first = FE_OK;
    for (int k = 0; k < count; ++k) {
        memset(&rs[k], 0, sizeof(fe_result));
        int rc = validate(ctx, &ps[k]);
        Slot *s = nullptr;
        if (rc == FE_OK) rc = acquire_slot(ctx, static_cast<int>(ps[k].n), slot_method(&ps[k]), &s);
        if (rc != FE_OK) {
            rs[k].status = rc;
            if (first == FE_OK) first = rc;
            continue;
        }
        jobs.push_back(make_job(&ps[k], s));
        idx.push_back(k);
    }
    if (!jobs.empty()) {
        std::vector<fe_result> tmp(jobs.size());
        const int rc = run_problems(ctx, jobs, tmp.data());
        for (size_t q = 0; q < jobs.size(); ++q) {
            rs[idx[q]] = tmp[q];
            release_slot(ctx, jobs[q].slot);
        }
        if (first == FE_OK) first = rc;
    }
    return first;
}

extern "C" int fe_submit(fe_ctx *ctx, const fe_problem *p, fe_ticket *t) {
    if (!ctx || !t) return set_err(nullptr, FE_EINVAL, "ctx or ticket pointer is NULL");
    *t = 0;
    int rc = validate(ctx, p);
    if (rc != FE_OK) return rc;
    const int n = static_cast<int>(p->n);
    const int method = slot_method(p);
    {
        int a, b, c;
        size_t np;
        if (slot_bytes(n, method, &a, &b, &c, &np) > ctx->budget)
            return set_err(ctx, FE_ENOMEM, "problem needs more than the whole HBM budget");
    }
    {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        if (ctx->stop) return set_err(ctx, FE_EINVAL, "context is shutting down");
        if (ctx->reqs.size() >= kMaxTickets) return set_err(ctx, FE_EBUSY, "too many outstanding tickets");
    }
    cudaSetDevice(ctx->device);
    Req *r = new Req();
    r->p = *p;
    r->t_submit = std::chrono::steady_clock::now();
    const bool dev = (p->flags & FE_PTR_DEVICE) != 0;
    const size_t row = sizeof(double) * n;
    Slot *s = nullptr;
    cudaError_t ce = cudaSuccess;
    if (acquire_slot(ctx, n, method, &s) == FE_OK) {
        // copy Hp straight into the slot
        ce = cudaMemcpy2DAsync(s->Hcopy, row, p->Hp, sizeof(double) * p->ld, row, n,
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->copy_stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->copy_stream);
        r->slot = s;
        r->staged = true;
    } else {
        // no room now: keep a host copy until a slot frees up
        r->hbuf.resize(static_cast<size_t>(n) * n);
        if (dev) {
            ce = cudaMemcpy2DAsync(r->hbuf.data(), row, p->Hp, sizeof(double) * p->ld, row, n,
                                   cudaMemcpyDeviceToHost, ctx->copy_stream);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->copy_stream);
        } else {
            for (int i = 0; i < n; ++i)
                memcpy(r->hbuf.data() + static_cast<size_t>(i) * n, p->Hp + static_cast<size_t>(i) * p->ld, row);
        }
    }
    if (ce != cudaSuccess) {
        if (r->slot) release_slot(ctx, r->slot);
        delete r;
        return cuda_fail(ctx, ce, "fe_submit copy of Hp");
    }
    r->p.Hp = nullptr;  // the caller's Hp is not referenced after this point
    {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        r->id = ctx->next_ticket++;
        ctx->reqs[r->id] = r;
        ctx->waiting.push_back(r);
        ctx->n_submitted += 1;
        if (!r->slot) {
            r->deferred = true;  // no room at submission: Hp waits in host memory
            ctx->n_deferred += 1;
        }
        ctx->peak_waiting = std::max<long long>(ctx->peak_waiting, static_cast<long long>(ctx->waiting.size()));
        if (!ctx->worker_started) {
            ctx->worker = std::thread(serve_loop, ctx);
            ctx->worker_started = true;
        }
        *t = r->id;
    }
    ctx->qcv.notify_one();
    return FE_OK;
}

extern "C" int fe_poll(fe_ctx *ctx, fe_ticket t, fe_result *r) {
    if (!ctx) return set_err(nullptr, FE_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->qmu);
    auto it = ctx->reqs.find(t);
    if (it == ctx->reqs.end()) return set_err(ctx, FE_EINVAL, "unknown ticket");
    Req *q = it->second;
    if (!q->done) return FE_PENDING;
    if (r) *r = q->res;
    const int status = q->res.status;
    ctx->reqs.erase(it);
    delete q;
    return status;
}

extern "C" const char *fe_last_error_string(const fe_ctx *) { return g_err.c_str(); }

int fe::set_error_string(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

// ============================================================== kernel-level entry points

extern "C" int fe_k_gershgorin(fe_ctx *ctx, const double *H, int64_t n, int64_t ld, double *out4) {
    if (!ctx || !H || !out4 || n < 1 || ld < n) return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    Engine &eg = ctx->eng;
    Slot *s = nullptr;
    int rc = acquire_slot(ctx, static_cast<int>(n), kMethodSp2, &s);
    if (rc != FE_OK) return rc;
    MmaProb hp = s->hp;
    hp.H = H;
    hp.ldh = ld;
    SolveState st0;
    memset(&st0, 0, sizeof(st0));
    st0.n = static_cast<int>(n);
    rc = ensure_dev(ctx, &eg.d_probs, &eg.probs_cap, 1);
    if (rc != FE_OK) { release_slot(ctx, s); return rc; }
    cudaStream_t q = eg.stream;
    SolveState res;
    cudaMemcpyAsync(eg.d_probs, &hp, sizeof(MmaProb), cudaMemcpyHostToDevice, q);
    cudaMemcpyAsync(s->st, &st0, sizeof(SolveState), cudaMemcpyHostToDevice, q);
    cudaMemsetAsync(s->bad, 0, sizeof(int), q);
    k_bounds_rows<<<ceil_div(static_cast<int>(n), 8), 256, 0, q>>>(eg.d_probs, 0, s->rowinfo, s->bad);
    k_bounds_reduce<<<1, 1024, 0, q>>>(eg.d_probs, 0, s->rowinfo, s->bad);
    ctx->launches += 2;
    cudaMemcpyAsync(&res, s->st, sizeof(SolveState), cudaMemcpyDeviceToHost, q);
    const cudaError_t e = cudaStreamSynchronize(q);
    release_slot(ctx, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gershgorin");
    out4[0] = res.emin;
    out4[1] = res.emax;
    out4[2] = res.trH;
    out4[3] = res.bad_input ? 1.0 : 0.0;
    return FE_OK;
}

extern "C" int fe_k_sym_square(fe_ctx *ctx, const float *Y, int64_t n, int64_t ldy, float *C,
                               int64_t ldc, int nslices, double bound) {
    if (!ctx || !Y || !C || n < 1 || ldy < n || ldc < n || (nslices != 1 && nslices != 2) ||
        !(bound > 0.0))
        return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    Engine &eg = ctx->eng;
    Slot *s = nullptr;
    int rc = acquire_slot(ctx, static_cast<int>(n), kMethodSp2, &s);
    if (rc != FE_OK) return rc;
    cudaStream_t q = eg.stream;
    int e2;
    frexp(bound, &e2);
    const float scale = static_cast<float>(ldexp(1.0, 14 - e2));
    // master <- Y (the epilogue then overwrites it with 1 * Y^2)
    cudaMemcpy2DAsync(s->Y, sizeof(float) * s->ldy, Y, sizeof(float) * ldy, sizeof(float) * n, n,
                      cudaMemcpyDeviceToDevice, q);
    k_make_slices<<<kInitBlocks, 256, 0, q>>>(s->Y, static_cast<int>(n), s->ldy, scale,
                                              s->hp.mats[kMatY0].sl[0], s->hp.mats[kMatY0].sl[1], s->lds);
    SolveState st0;
    memset(&st0, 0, sizeof(st0));
    st0.n = static_cast<int>(n);
    st0.kind = (nslices == 2) ? kTcSplit : kTcSingle;
    // one output: master of slot 0 <- 1 * v + 0 * Y, slices of slot 1 (unused) at scale 1
    ProdOp &op = st0.op;
    op.A = op.B = kMatY0;
    op.E1 = kMatY0;
    op.E2 = -1;
    op.inv = static_cast<float>(1.0 / (static_cast<double>(scale) * scale));
    op.nout = 1;
    op.part_out = 0;
    op.out[0].mat = kMatY1;
    op.out[0].flags = kOutMaster | kOutSlices;
    op.out[0].a = 1.0f;
    op.out[0].s = 1.0f;
    // tile width from the context's table for this n (split: FE_PREC_FP32, single: FE_PREC_TRY_FP16)
    const int bn = tile_width(ctx, n, nslices == 2 ? FE_PREC_FP32 : FE_PREC_TRY_FP16);
    const std::vector<TileEnt> &tl = (bn == kTileM) ? s->tilesN : s->tiles;
    rc = ensure_dev(ctx, &eg.d_probs, &eg.probs_cap, 1);
    if (rc == FE_OK) rc = ensure_dev(ctx, &eg.d_tiles, &eg.tiles_cap, tl.size());
    if (rc != FE_OK) { release_slot(ctx, s); return rc; }
    MmaProb hp = s->hp;
    hp.tc_tile0 = 0;
    hp.tc_ntiles = static_cast<int>(tl.size());
    hp.ntiles = static_cast<int>(tl.size());
    hp.bn = bn;
    cudaMemcpyAsync(eg.d_probs, &hp, sizeof(MmaProb), cudaMemcpyHostToDevice, q);
    cudaMemcpyAsync(eg.d_tiles, tl.data(), sizeof(TileEnt) * tl.size(), cudaMemcpyHostToDevice, q);
    cudaMemsetAsync(eg.d_skcnt, 0, sizeof(int) * 2 * ctx->num_sms, q);
    cudaMemcpyAsync(s->st, &st0, sizeof(SolveState), cudaMemcpyHostToDevice, q);
    cudaMemsetAsync(eg.d_err, 0, sizeof(int), q);
    const int nt = static_cast<int>(tl.size());
    k_sym_mma<<<ctx->num_sms, kSymThreads, mma_smem_bytes(), q>>>(eg.d_probs, 1, eg.d_tiles, nt, eg.d_err,
                                                                   eg.d_skws, eg.d_skcnt);
    ctx->launches += 2;
    cudaMemcpy2DAsync(C, sizeof(float) * ldc, s->Y, sizeof(float) * s->ldy, sizeof(float) * n, n,
                      cudaMemcpyDeviceToDevice, q);
    int herr = 0;
    cudaMemcpyAsync(&herr, eg.d_err, sizeof(int), cudaMemcpyDeviceToHost, q);
    const cudaError_t e = cudaStreamSynchronize(q);
    release_slot(ctx, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sym_square");
    if (herr) return set_err(ctx, FE_ETIMEOUT, "device wait timed out (code " + std::to_string(herr) + ")");
    return FE_OK;
}

extern "C" int fe_k_digit_square(fe_ctx *ctx, const double *X, int64_t n, int64_t ld, double *P,
                                 int64_t ldp) {
    if (!ctx || !X || !P || n < 1 || ld < n || ldp < n) return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    Engine &eg = ctx->eng;
    Slot *s = nullptr;
    int rc = acquire_slot(ctx, static_cast<int>(n), kMethodSp2, &s);
    if (rc != FE_OK) return rc;
    rc = ensure_dev(ctx, &eg.d_probs, &eg.probs_cap, 1);
    if (rc == FE_OK) rc = ensure_dev(ctx, &eg.d_tilesD, &eg.tilesD_cap, s->tilesD.size());
    if (rc != FE_OK) { release_slot(ctx, s); return rc; }
    cudaStream_t q = eg.stream;
    // input X as the FP64 iterate; one X^2 step with gamma = 0 writes X^2 to the other buffer
    cudaMemcpy2DAsync(s->Xd[0], sizeof(double) * s->ldx, X, sizeof(double) * ld, sizeof(double) * n, n,
                      cudaMemcpyDeviceToDevice, q);
    SolveState st0;
    memset(&st0, 0, sizeof(st0));
    st0.n = static_cast<int>(n);
    st0.kind = kDigit;
    st0.x_fp64 = 1;
    st0.xcur = 0;
    st0.sq = 1;
    MmaProb hp = s->hp;
    hp.H = X;
    hp.ldh = ld;
    cudaMemcpyAsync(eg.d_probs, &hp, sizeof(MmaProb), cudaMemcpyHostToDevice, q);
    cudaMemcpyAsync(eg.d_tilesD, s->tilesD.data(), sizeof(TileEnt) * s->tilesD.size(),
                    cudaMemcpyHostToDevice, q);
    cudaMemcpyAsync(s->st, &st0, sizeof(SolveState), cudaMemcpyHostToDevice, q);
    cudaMemsetAsync(eg.d_err, 0, sizeof(int), q);
    const int nt = static_cast<int>(s->tilesD.size());
    k_digit_prep<<<2 * ctx->num_sms, 256, 0, q>>>(eg.d_probs, 1);
    k_digit_mma<<<std::min(nt, ctx->num_sms), kMmaThreads, digit_smem_bytes(), q>>>(eg.d_probs, eg.d_tilesD,
                                                                                    nt, eg.d_err);
    ctx->launches += 2;
    cudaMemcpy2DAsync(P, sizeof(double) * ldp, s->Xd[1], sizeof(double) * s->ldx, sizeof(double) * n, n,
                      cudaMemcpyDeviceToDevice, q);
    int herr = 0;
    cudaMemcpyAsync(&herr, eg.d_err, sizeof(int), cudaMemcpyDeviceToHost, q);
    const cudaError_t e = cudaStreamSynchronize(q);
    release_slot(ctx, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "digit_square");
    if (herr) return set_err(ctx, FE_ETIMEOUT, "device wait timed out (code " + std::to_string(herr) + ")");
    return FE_OK;
}

// ============================================================== either side of the expansion

namespace {

// Run C = A B^T (k_gemm_split, + k_gemm_reduce in split mode) on the
// context's stream with the slices already in the workspace; blocking.
int run_gemm(fe_ctx *ctx, const GemmArgs &ga, const std::vector<TileEnt> &tl, const char *what) {
    Engine &eg = ctx->eng;
    cudaStream_t q = eg.stream;
    int rc = ensure_dev(ctx, &ctx->d_gtiles, &ctx->gtiles_cap, tl.size());
    if (rc != FE_OK) return rc;
    FE_CUDA(ctx, cudaMemcpyAsync(ctx->d_gargs, &ga, sizeof(GemmArgs), cudaMemcpyHostToDevice, q));
    FE_CUDA(ctx, cudaMemcpyAsync(ctx->d_gtiles, tl.data(), sizeof(TileEnt) * tl.size(), cudaMemcpyHostToDevice, q));
    FE_CUDA(ctx, cudaMemsetAsync(eg.d_err, 0, sizeof(int), q));
    const int units = ga.ntiles * (ga.nsplit > 0 ? ga.nsplit : 1);
    FE_CUDA(ctx, cudaEventRecord(eg.ev_setup, q));
    k_gemm_split<<<std::min(units, ctx->num_sms), kGemmThreads, gemm_smem_bytes(), q>>>(ctx->d_gargs, ctx->d_gtiles,
                                                                                        eg.d_err);
    ctx->launches += 1;
    FE_CUDA(ctx, cudaEventRecord(eg.ev_loop, q));
    if (ga.nsplit > 0) {
        k_gemm_reduce<<<ga.ntiles, 256, 0, q>>>(ctx->d_gargs, ctx->d_gtiles);
        ctx->launches += 1;
    }
    FE_CUDA(ctx, cudaEventRecord(eg.ev1, q));
    FE_CUDA(ctx, cudaGetLastError());
    int herr = 0;
    FE_CUDA(ctx, cudaMemcpyAsync(&herr, eg.d_err, sizeof(int), cudaMemcpyDeviceToHost, q));
    const cudaError_t e = cudaStreamSynchronize(q);
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    // operand split, tensor-core product, reduction of the K parts
    float a = 0.0f, b = 0.0f, c = 0.0f;
    cudaEventElapsedTime(&a, eg.ev0, eg.ev_setup);
    cudaEventElapsedTime(&b, eg.ev_setup, eg.ev_loop);
    cudaEventElapsedTime(&c, eg.ev_loop, eg.ev1);
    ctx->phase_ms[0] = a;
    ctx->phase_ms[1] = b;
    ctx->phase_ms[2] = c;
    ctx->phase_ms[3] = units;
    if (herr) return set_err(ctx, FE_ETIMEOUT, std::string(what) + ": device wait timed out (code " +
                                                   std::to_string(herr) + ")");
    return FE_OK;
}

// Workspace of `bytes` and the small device blocks of the GEMM path.
int gemm_workspace(fe_ctx *ctx, size_t bytes) {
    if (!ctx->d_gargs) FE_CUDA(ctx, cudaMalloc(&ctx->d_gargs, sizeof(GemmArgs)));
    if (!ctx->d_amax) FE_CUDA(ctx, cudaMalloc(&ctx->d_amax, 2 * sizeof(unsigned long long)));
    if (bytes <= ctx->gws_cap) return FE_OK;
    if (ctx->gws) cudaFree(ctx->gws);
    ctx->gws = nullptr;
    ctx->gws_cap = 0;
    if (bytes > ctx->budget) return set_err(ctx, FE_ENOMEM, "workspace of " + std::to_string(bytes) +
                                                                 " bytes exceeds the HBM budget");
    if (cudaMalloc(&ctx->gws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, FE_ENOMEM, "no device memory for the workspace");
    }
    ctx->gws_cap = bytes;
    return FE_OK;
}

// Blocks of k_split_rows: one per row (direct) or per 64 x 64 tile
// (transposed), at most 8 per SM (the kernel loops).
int split_grid(fe_ctx *ctx, int64_t rows, int64_t cols, bool transpose) {
    const int64_t t = transpose ? ((rows + 63) / 64) * ((cols + 63) / 64) : rows;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(t, 8LL * ctx->num_sms)));
}

}  // namespace

extern "C" int fe_project(fe_ctx *ctx, const double *Psi, const double *HPsi, int64_t m, int64_t n, int64_t ld,
                          double *Hp, int64_t ldh) {
    if (!ctx) return set_err(nullptr, FE_EINVAL, "ctx is NULL");
    if (!Psi || !HPsi || !Hp || m < 1 || n < 1 || n > (1 << 20) || m > INT_MAX || ld < n || ldh < n)
        return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t q = ctx->eng.stream;
    const int64_t lds = static_cast<int64_t>(align_up(static_cast<size_t>(m), 8));  // slices of Psi^T: n rows of m
    const int nk = static_cast<int>((m + kTileK - 1) / kTileK);
    // upper-triangle tiles: 128-row block I, 192-column panel J holding some j >= i
    std::vector<TileEnt> tl;
    const int TI = static_cast<int>((n + kTileM - 1) / kTileM), TJ = static_cast<int>((n + kGemmN - 1) / kGemmN);
    for (int J = 0; J < TJ; ++J)
        for (int I = 0; I < TI; ++I)
            if (static_cast<int64_t>(J) * kGemmN + kGemmN - 1 >= static_cast<int64_t>(I) * kTileM)
                tl.push_back(TileEnt{0, I, J, 0});
    const int ntiles = static_cast<int>(tl.size());
    // K parts: at most 128 chunks (K = 8192) summed in FP32 per part, and
    // enough work units for about six waves over the SMs; at least 8 chunks a part
    int S = std::max((nk + 127) / 128, (6 * ctx->num_sms + ntiles - 1) / ntiles);
    S = std::max(1, std::min(S, std::max(1, nk / 8)));
    const int cs = (nk + S - 1) / S;
    S = (nk + cs - 1) / cs;  // every part non-empty
    const size_t slice = 2 * static_cast<size_t>(n) * static_cast<size_t>(lds);
    const size_t tsz = static_cast<size_t>(kTileM) * kGemmN * sizeof(float);
    const size_t bytes = align_up(4 * slice, 1024) + static_cast<size_t>(ntiles) * S * tsz;
    int rc = gemm_workspace(ctx, bytes);
    if (rc != FE_OK) return rc;
    __half *sl[4];
    for (int k = 0; k < 4; ++k) sl[k] = reinterpret_cast<__half *>(ctx->gws + k * slice);
    GemmArgs ga;
    memset(&ga, 0, sizeof(ga));
    for (int k = 0; k < 2 && rc == FE_OK; ++k) {
        rc = encode_map_rect(ctx, &ga.tA[k], sl[k], m, n, lds, kTileM);
        if (rc == FE_OK) rc = encode_map_rect(ctx, &ga.tB[k], sl[2 + k], m, n, lds, kGemmN);
    }
    if (rc != FE_OK) return rc;
    ga.C = Hp;
    ga.ldc = ldh;
    ga.ws = reinterpret_cast<float *>(ctx->gws + align_up(4 * slice, 1024));
    ga.amax = ctx->d_amax;
    ga.rows_a = ga.rows_b = static_cast<int>(n);
    ga.kdim = static_cast<int>(m);
    ga.nsplit = S;
    ga.ntiles = ntiles;
    FE_CUDA(ctx, cudaEventRecord(ctx->eng.ev0, q));
    FE_CUDA(ctx, cudaMemsetAsync(ctx->d_amax, 0, 2 * sizeof(unsigned long long), q));
    k_absmax<<<4 * ctx->num_sms, 256, 0, q>>>(Psi, m, n, ld, ctx->d_amax);
    k_absmax<<<4 * ctx->num_sms, 256, 0, q>>>(HPsi, m, n, ld, ctx->d_amax + 1);
    const int gs = split_grid(ctx, m, n, true);
    k_split_rows<<<gs, 256, 0, q>>>(Psi, m, n, ld, ctx->d_amax, sl[0], sl[1], lds, 1);
    k_split_rows<<<gs, 256, 0, q>>>(HPsi, m, n, ld, ctx->d_amax + 1, sl[2], sl[3], lds, 1);
    ctx->launches += 4;
    return run_gemm(ctx, ga, tl, "fe_project");
}

extern "C" int fe_rotate(fe_ctx *ctx, const double *Psi, int64_t m, int64_t n, int64_t ldpsi, const double *D,
                         int64_t ldd, double *Out, int64_t ldo) {
    if (!ctx) return set_err(nullptr, FE_EINVAL, "ctx is NULL");
    if (!Psi || !D || !Out || m < 1 || n < 1 || n > (1 << 20) || m > INT_MAX || ldpsi < n || ldd < n || ldo < n)
        return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t q = ctx->eng.stream;
    const int64_t lds = static_cast<int64_t>(align_up(static_cast<size_t>(n), 8));  // K = n
    std::vector<TileEnt> tl;
    const int TI = static_cast<int>((m + kTileM - 1) / kTileM), TJ = static_cast<int>((n + kGemmN - 1) / kGemmN);
    for (int I = 0; I < TI; ++I)
        for (int J = 0; J < TJ; ++J) tl.push_back(TileEnt{0, I, J, 0});
    const size_t sa = 2 * static_cast<size_t>(m) * static_cast<size_t>(lds);
    const size_t sb = 2 * static_cast<size_t>(n) * static_cast<size_t>(lds);
    const size_t oa = align_up(sa, 1024), ob = align_up(sb, 1024);
    int rc = gemm_workspace(ctx, 2 * oa + 2 * ob);
    if (rc != FE_OK) return rc;
    __half *ah = reinterpret_cast<__half *>(ctx->gws), *al = reinterpret_cast<__half *>(ctx->gws + oa);
    __half *bh = reinterpret_cast<__half *>(ctx->gws + 2 * oa), *bl = reinterpret_cast<__half *>(ctx->gws + 2 * oa + ob);
    GemmArgs ga;
    memset(&ga, 0, sizeof(ga));
    rc = encode_map_rect(ctx, &ga.tA[0], ah, n, m, lds, kTileM);
    if (rc == FE_OK) rc = encode_map_rect(ctx, &ga.tA[1], al, n, m, lds, kTileM);
    if (rc == FE_OK) rc = encode_map_rect(ctx, &ga.tB[0], bh, n, n, lds, kGemmN);
    if (rc == FE_OK) rc = encode_map_rect(ctx, &ga.tB[1], bl, n, n, lds, kGemmN);
    if (rc != FE_OK) return rc;
    ga.C = Out;
    ga.ldc = ldo;
    ga.amax = ctx->d_amax;
    ga.rows_a = static_cast<int>(m);
    ga.rows_b = static_cast<int>(n);
    ga.kdim = static_cast<int>(n);
    ga.nsplit = 0;
    ga.ntiles = static_cast<int>(tl.size());
    FE_CUDA(ctx, cudaEventRecord(ctx->eng.ev0, q));
    FE_CUDA(ctx, cudaMemsetAsync(ctx->d_amax, 0, 2 * sizeof(unsigned long long), q));
    k_absmax<<<4 * ctx->num_sms, 256, 0, q>>>(Psi, m, n, ldpsi, ctx->d_amax);
    k_absmax<<<4 * ctx->num_sms, 256, 0, q>>>(D, n, n, ldd, ctx->d_amax + 1);
    k_split_rows<<<split_grid(ctx, m, n, false), 256, 0, q>>>(Psi, m, n, ldpsi, ctx->d_amax, ah, al, lds, 0);
    k_split_rows<<<split_grid(ctx, n, n, false), 256, 0, q>>>(D, n, n, ldd, ctx->d_amax + 1, bh, bl, lds, 0);
    ctx->launches += 4;
    return run_gemm(ctx, ga, tl, "fe_rotate");
}

extern "C" int fe_k_profile(fe_ctx *ctx, int enable) {
    if (!ctx) return set_err(nullptr, FE_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->prof = enable != 0;
    return FE_OK;
}

extern "C" int fe_k_serve_stats(fe_ctx *ctx, int64_t *out4, int reset) {
    if (!ctx || !out4) return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(ctx->qmu);
    out4[0] = ctx->n_submitted;
    out4[1] = ctx->n_deferred;
    out4[2] = ctx->peak_waiting;
    out4[3] = ctx->peak_running;
    if (reset) ctx->n_submitted = ctx->n_deferred = ctx->peak_waiting = ctx->peak_running = 0;
    return FE_OK;
}

extern "C" int fe_k_set_wait(fe_ctx *ctx, double limit_ms, int fail_partner) {
    if (!ctx) return set_err(nullptr, FE_EINVAL, "ctx is NULL");
    if (!(limit_ms > 0.0 && limit_ms <= 60000.0)) return set_err(ctx, FE_EINVAL, "limit_ms must be in (0, 60000]");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    DevCtl c{};
    c.fail_partner = fail_partner ? 1 : 0;
    c.wait_ns = static_cast<unsigned long long>(limit_ms * 1e6);
    for (Engine *e : {&ctx->eng, &ctx->seng}) {
        // every field after the error word; the streams order it after earlier work
        FE_CUDA(ctx, cudaMemcpyAsync(reinterpret_cast<char *>(e->d_err) + sizeof(int),
                                     reinterpret_cast<const char *>(&c) + sizeof(int), sizeof(DevCtl) - sizeof(int),
                                     cudaMemcpyHostToDevice, e->stream));
        FE_CUDA(ctx, cudaStreamSynchronize(e->stream));
    }
    return FE_OK;
}

extern "C" int fe_k_profile_kinds(fe_ctx *ctx, double *ms8, int *n8) {
    if (!ctx || !ms8 || !n8) return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (int q = 0; q < 8; ++q) {
        ms8[q] = ctx->prof_kind_ms[q];
        n8[q] = ctx->prof_kind_n[q];
    }
    return FE_OK;
}

extern "C" int fe_k_narrow_bounds(fe_ctx *ctx, double factor) {
    if (!ctx) return set_err(nullptr, FE_EINVAL, "ctx is NULL");
    if (!(factor > 0.0 && factor <= 1.0)) return set_err(ctx, FE_EINVAL, "factor must be in (0, 1]");
    ctx->lz_narrow.store(factor, std::memory_order_relaxed);
    return FE_OK;
}

extern "C" int fe_k_profile_steps(fe_ctx *ctx, double *out, int max_steps, int *count) {
    if (!ctx || !out || !count || max_steps < 0) return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    const int m = std::min(max_steps, static_cast<int>(ctx->prof_steps.size()));
    for (int i = 0; i < m; ++i) out[i] = ctx->prof_steps[i];
    *count = m;
    return FE_OK;
}

extern "C" int fe_k_phase_ms(fe_ctx *ctx, double *out4) {
    if (!ctx || !out4) return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (int i = 0; i < 4; ++i) out4[i] = ctx->phase_ms[i];
    return FE_OK;
}

extern "C" int fe_k_profile_read(fe_ctx *ctx, double *out8) {
    if (!ctx || !out8) return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (int i = 0; i < 8; ++i) out8[i] = ctx->prof_out[i];
    return FE_OK;
}

extern "C" int fe_k_launch_count(fe_ctx *ctx, int64_t *out) {
    if (!ctx || !out) return set_err(ctx, FE_EINVAL, "bad arguments");
    *out = ctx->launches.load();
    return FE_OK;
}

extern "C" int fe_k_history(fe_ctx *ctx, int index, double *out, int max_rows, int *rows) {
    if (!ctx || !out || !rows || max_rows < 0 || index < 0) return set_err(ctx, FE_EINVAL, "bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    const Engine &eg = ctx->eng;
    if (!eg.h_states || static_cast<size_t>(index) >= eg.h_states_cap)
        return set_err(ctx, FE_EINVAL, "no such problem in the last solve");
    const SolveState &st = eg.h_states[index];
    const int r = std::min({st.iter + 1, kHistRows, max_rows});
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < kHistCols; ++j) out[i * kHistCols + j] = st.hist[i][j];
    *rows = r;
    return FE_OK;
}

extern "C" int fe_autotune(fe_ctx *ctx, int count, const int64_t *ns, uint32_t prec, int reps, fe_tune *out) {
    if (!ctx || count < 0 || (count > 0 && !ns)) return set_err(ctx, FE_EINVAL, "bad arguments");
    if ((prec & ~FE_PREC_MASK) != 0) return set_err(ctx, FE_EINVAL, "unknown precision flag");
    if (prec == 0) prec = ctx->prec_default & FE_PREC_MASK;
    if (prec != FE_PREC_MIXED && prec != FE_PREC_FP32 && prec != FE_PREC_TRY_FP16)
        return set_err(ctx, FE_EINVAL, "only the tensor-core schedules (MIXED, FP32, TRY_FP16) have tiles to tune");
    if (reps < 1) reps = 2;
    // the largest n given for each panel count is the one timed
    std::map<int, int64_t> Tn;
    for (int i = 0; i < count; ++i) {
        if (ns[i] < 2 || ns[i] > (1 << 20)) return set_err(ctx, FE_EINVAL, "n out of range (2 .. 2^20)");
        const int T = static_cast<int>((ns[i] + kTileM - 1) / kTileM);
        Tn[T] = std::max(Tn[T], ns[i]);
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t q = ctx->eng.stream;
    for (const auto &tn : Tn) {
        const int T = tn.first;
        const int64_t n = tn.second;
        // synthetic gapped Hp: diagonal, N_e = round(0.85 n) levels evenly in
        // [-1, -0.05], the rest evenly in [0.05, 0.5] (the tensor-core work of a
        // product does not depend on the values)
        const int64_t ne = std::min<int64_t>(n - 1, std::max<int64_t>(1, llround(0.85 * static_cast<double>(n))));
        std::vector<double> diag(static_cast<size_t>(n));
        for (int64_t i = 0; i < n; ++i)
            diag[i] = (i < ne) ? -1.0 + 0.95 * static_cast<double>(i) / static_cast<double>(std::max<int64_t>(1, ne - 1))
                               : 0.05 + 0.45 * static_cast<double>(i - ne) / static_cast<double>(std::max<int64_t>(1, n - ne - 1));
        double *dH = nullptr;
        const size_t bytes = sizeof(double) * static_cast<size_t>(n) * static_cast<size_t>(n);
        if (cudaMalloc(&dH, bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_err(ctx, FE_ENOMEM, "autotune: no device memory for Hp");
        }
        int rc = FE_OK;
        if (cudaMemsetAsync(dH, 0, bytes, q) != cudaSuccess ||
            cudaMemcpy2DAsync(dH, sizeof(double) * static_cast<size_t>(n + 1), diag.data(), sizeof(double),
                              sizeof(double), static_cast<size_t>(n), cudaMemcpyHostToDevice, q) != cudaSuccess ||
            cudaStreamSynchronize(q) != cudaSuccess)
            rc = set_err(ctx, FE_ECUDA, std::string("autotune: ") + cudaGetErrorString(cudaGetLastError()));
        fe_problem p{};
        p.Hp = dH;
        p.n = n;
        p.ld = n;
        p.n_e = static_cast<double>(ne);
        p.flags = FE_PTR_DEVICE | FE_METHOD_SP2 | prec;
        // throughput, not latency: enough copies of the problem in one batch
        // for two waves of 128 x 256 tiles over the SMs (at most 16 copies;
        // they share the read-only Hp)
        const int wide_tiles = T * ((T + 1) / 2);
        const int copies = std::max(1, std::min(16, (2 * ctx->num_sms + wide_tiles - 1) / wide_tiles));
        std::vector<fe_problem> ps(copies, p);
        std::vector<fe_result> rs(copies);
        double best[2] = {DBL_MAX, DBL_MAX};
        // the entry before tuning, put back if a trial fails
        bool had = false;
        TuneEnt prev;
        {
            std::lock_guard<std::mutex> tl(ctx->tmu);
            auto it = ctx->tune.find({T, prec});
            if (it != ctx->tune.end()) {
                had = true;
                prev = it->second;
            }
        }
        // a warm-up batch per width (slots, graph), then `reps` rounds taking turns
        for (int r = 0; r <= reps && rc == FE_OK; ++r)
            for (int w = 0; w < 2 && rc == FE_OK; ++w) {
                {
                    std::lock_guard<std::mutex> tl(ctx->tmu);
                    ctx->tune[{T, prec}] = TuneEnt{w == 0 ? kTileN : kTileM, 0.0, 0.0};
                }
                rc = fe_solve_batch(ctx, copies, ps.data(), rs.data());
                double ms = 0.0;
                for (const fe_result &x : rs) ms = std::max(ms, x.ms);
                if (rc == FE_OK && r > 0) best[w] = std::min(best[w], ms / copies);
            }
        cudaFree(dH);
        std::lock_guard<std::mutex> tl(ctx->tmu);
        if (rc != FE_OK) {
            if (had) ctx->tune[{T, prec}] = prev;
            else ctx->tune.erase({T, prec});
            return rc;
        }
        ctx->tune[{T, prec}] = TuneEnt{best[1] < best[0] ? kTileM : kTileN, best[0], best[1]};
    }
    if (out)
        for (int i = 0; i < count; ++i) {
            const int T = static_cast<int>((ns[i] + kTileM - 1) / kTileM);
            std::lock_guard<std::mutex> tl(ctx->tmu);
            const TuneEnt &e = ctx->tune[{T, prec}];
            out[i].n = ns[i];
            out[i].bn = e.bn;
            out[i].ms_256 = e.ms_w;
            out[i].ms_128 = e.ms_n;
        }
    std::lock_guard<std::mutex> tl(ctx->tmu);
    return save_tune(ctx);
}

extern "C" int fe_autotune_batch(fe_ctx *ctx, int count, const fe_problem *ps, int reps, double *trial_ms,
                                 int max_trials, int *ntrials) {
    if (ntrials) *ntrials = 0;
    if (!ctx || count < 1 || !ps || max_trials < 0 || (max_trials > 0 && !trial_ms))
        return set_err(ctx, FE_EINVAL, "bad arguments");
    if (reps < 1) reps = 2;
    for (int k = 0; k < count; ++k) {
        const int rc = validate(ctx, &ps[k]);
        if (rc != FE_OK) return rc;
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    // the batch's tile classes (panel count, policy), smallest first
    std::vector<std::pair<int, uint32_t>> cls;
    for (int k = 0; k < count; ++k) {
        const uint32_t pr = prec_of(ctx, &ps[k]);
        if (pr == FE_PREC_FP64 && method_of(&ps[k]) != kMethodFermi) continue;
        cls.push_back({static_cast<int>((ps[k].n + kTileM - 1) / kTileM), pr});
    }
    std::sort(cls.begin(), cls.end());
    cls.erase(std::unique(cls.begin(), cls.end()), cls.end());
    if (cls.empty()) return FE_OK;
    std::map<std::pair<int, uint32_t>, TuneEnt> saved;
    {
        std::lock_guard<std::mutex> tl(ctx->tmu);
        for (const auto &c : cls) {
            auto it = ctx->tune.find(c);
            if (it != ctx->tune.end()) saved[c] = it->second;
            ctx->tune[c] = TuneEnt{kTileN, 0.0, 0.0};
        }
    }
    // the batch without its outputs
    std::vector<fe_problem> q(ps, ps + count);
    for (fe_problem &x : q) x.D = nullptr;
    std::vector<fe_result> rs(count);
    auto time_batch = [&](double *out) {
        double best = DBL_MAX;
        for (int r = 0; r <= reps; ++r) {  // the first run builds slots and the graph
            const int rc = fe_solve_batch(ctx, count, q.data(), rs.data());
            if (rc != FE_OK) return rc;
            double ms = 0.0;
            for (const fe_result &x : rs) ms = std::max(ms, x.ms);
            if (r > 0) best = std::min(best, ms);
        }
        *out = best;
        return FE_OK;
    };
    auto set_bn = [&](const std::pair<int, uint32_t> &c, int bn) {
        std::lock_guard<std::mutex> tl(ctx->tmu);
        ctx->tune[c] = TuneEnt{bn, 0.0, 0.0};
    };
    int nt = 0;
    auto log = [&](double ms) {
        if (nt < max_trials) trial_ms[nt] = ms;
        ++nt;
    };
    double best = 0.0;
    int rc = time_batch(&best);
    if (rc == FE_OK) log(best);
    // narrow tiles for the smallest classes, one class more per trial, while
    // the batch gets faster (by more than 0.5%)
    for (size_t c = 0; c < cls.size() && rc == FE_OK; ++c) {
        set_bn(cls[c], kTileM);
        double ms = 0.0;
        rc = time_batch(&ms);
        if (rc != FE_OK) break;
        log(ms);
        if (ms < best * 0.995) {
            best = ms;
        } else {
            set_bn(cls[c], kTileN);
            break;
        }
    }
    if (ntrials) *ntrials = nt;
    std::lock_guard<std::mutex> tl(ctx->tmu);
    if (rc != FE_OK) {
        for (const auto &c : cls) {
            auto it = saved.find(c);
            if (it != saved.end()) ctx->tune[c] = it->second;
            else ctx->tune.erase(c);
        }
        return rc;
    }
    return save_tune(ctx);
}

extern "C" int fe_k_set_tile_width(fe_ctx *ctx, int64_t n, uint32_t prec, int bn) {
    if (!ctx || n < 1 || (prec & ~FE_PREC_MASK) != 0 || (bn != 0 && bn != kTileM && bn != kTileN))
        return set_err(ctx, FE_EINVAL, "bad arguments");
    const int T = static_cast<int>((n + kTileM - 1) / kTileM);
    std::lock_guard<std::mutex> tl(ctx->tmu);
    if (bn == 0) ctx->tune.erase({T, prec});
    else ctx->tune[{T, prec}] = TuneEnt{bn, 0.0, 0.0};
    return FE_OK;
}

extern "C" int fe_k_tile_width(fe_ctx *ctx, int64_t n, uint32_t prec, int *bn) {
    if (!ctx || !bn || n < 1 || (prec & ~FE_PREC_MASK) != 0) return set_err(ctx, FE_EINVAL, "bad arguments");
    *bn = tile_width(ctx, n, prec);
    return FE_OK;
}
