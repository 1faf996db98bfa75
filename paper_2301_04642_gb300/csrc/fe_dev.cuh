// Device-side definitions shared by the kernels of the Fermi-operator
// expansion library (sm_103a).
//
// Representation of the SP2 iterate (Sec. II-B1, Eq. (1)): X = c I + Y with the
// scalar shift c kept in FP64 and Y stored as an FP32 master matrix.  The
// tensor-core products read Y through FP16 "slices" scaled by a power of two s:
//   s Y ~= hi + lo,  hi = fp16(s Y),  lo = fp16(s Y - hi)
// so Y^2 ~= (hi hi^T + hi lo^T + lo hi^T) / s^2 accumulated in FP32 (TMEM).
// With X = c I + Y an SP2 step becomes an update of (c, Y):
//   X^2      -> c' = c^2,        Y' = 2c Y + Y^2
//   2X - X^2 -> c' = 2c - c^2,   Y' = (2 - 2c) Y - Y^2
// (Sec. II-B1: "X_{n+1} = X_n +/- (X_n - X_n^2)").
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace fe {

// ---------------------------------------------------------------- constants
constexpr int kTileM = 128;    // rows of one tensor-core tile (TMEM lanes)
constexpr int kTileN = 256;    // columns of one tensor-core tile (two 128-blocks)
constexpr int kTileK = 64;     // K per pipeline stage (one 128-byte swizzle row of FP16)
constexpr int kMaxSlices = 2;
constexpr int kStages = 2;
constexpr int kSliceABytes = kTileM * kTileK * 2;   // 16 KiB
constexpr int kSliceBBytes = kTileN * kTileK * 2;   // 32 KiB
constexpr int kStageBytes = kMaxSlices * (kSliceABytes + kSliceBBytes);  // 96 KiB
constexpr int kMmaThreads = 320;  // digit kernel: warp 0 TMA, warp 1 MMA, warps 2-9 drain + epilogue
constexpr int kEpiWarps = 8;
// split-FP16 kernel: warpgroup 0 (warp 0 TMA, warp 1 MMA, warps 2-3 idle) gives
// registers to warpgroups 1-2 (8 drain + epilogue warps) with setmaxnreg.
// The launch gives every thread kSymLaunchRegs (384 threads: at most 3 warps
// per SM sub-partition of 16384 registers -> 168); 128 x 40 + 256 x 232 =
// 384 x 168, so the increase never waits for registers that are not there.
constexpr int kSymThreads = 384;
constexpr int kSymEpiWarp0 = 4;
constexpr int kSymLaunchRegs = 168;
constexpr int kSymRegsLow = 40;
constexpr int kSymRegsHigh = 232;
static_assert(128 * kSymRegsLow + 256 * kSymRegsHigh == kSymThreads * kSymLaunchRegs,
              "register split must equal the launch allocation");
constexpr int kPartStride = 4;    // doubles per partial slot: tr, sumsq, maxabs, spare
constexpr float kSliceTop = 16384.0f;  // slices are scaled so |s Y| <= 2^14 < fp16 max

// FP64-accurate products on the tensor cores (kind kDigit): X/4 is written in
// fixed point as kDigits balanced base-256 digits S_a in [-128, 127], each held
// exactly in FP16, X/4 = sum_a S_a 2^(-8(a+1)).  Level L of the product
// collects the digit pairs a + c = L; per K block of kDigitKBlock its integer
// sum is below 7 * 128 * 2^14 < 2^24, so the FP32 accumulator is exact.
constexpr int kDigits = 7;
constexpr int kDigitN = 64;       // tile columns (7 level buffers x 64 TMEM columns)
constexpr int kDigitK = 32;       // K per pipeline stage (one 64-byte swizzle row of FP16)
constexpr int kDigitStages = 2;   // 2 x 84 KiB (4 x 42 KiB stages of K = 16 measured slower)
constexpr int kDigitKBlock = 128; // K per drain of the level buffers

// error codes written by kernels into the context's device error word
enum DevErr : int {
    kErrNone = 0,
    kErrTimeoutFull = 1,    // TMA data never arrived
    kErrTimeoutEmpty = 2,   // smem stage never released
    kErrTimeoutTmem = 3,    // accumulator hand-off never happened
    kErrBadInput = 4,
    kErrTimeoutPartner = 5, // the partial sums of a split tile never arrived
    kErrTimeoutGrid = 6,    // a grid barrier of a cooperative launch never completed
};

// bounded waits give up after this many nanoseconds of wall time unless the
// context sets another limit (DevCtl::wait_ns)
constexpr uint64_t kWaitTimeoutNs = 2000000000ull;

// Device control block of one engine, passed to the kernels that wait: the
// first error code of the run (the host clears it before each run), the
// limit of every bounded wait, the arrival counter of the grid barriers of
// the cooperative Lanczos launch (zeroed before it), and a test hook.  With
// fail_partner set, the
// wait of the second CTA of a split tile in k_sym_mma watches `never` (a word
// nothing writes) instead of its partner's flag, so the wait runs out, the
// kernel records kErrTimeoutPartner and returns; it exists to test that
// expiry path.
struct DevCtl {
    int err;
    int fail_partner;
    int never;
    int pad;
    unsigned long long wait_ns;
    unsigned lz_bar;
    unsigned pad2;
};

constexpr int kHistRows = 160;  // per-step history kept in the solve state
constexpr int kLanczosSteps = 12;   // Lanczos steps of the spectral-bound estimate
constexpr int kCheckSteps = 3;      // logistic steps certifying the estimate (T_8)
constexpr int kStatusEscaped = -100;  // internal: an eigenvalue left [0, 1] (bounds too tight)
constexpr int kStatusAccelFailed = -101;  // internal: HOMO/LUMO estimates inconsistent (run plain SP2)
constexpr int kTrfoeMaxSteps = 128;   // branch bits kept for the truncated expansion
constexpr int kKindLog = 768;         // per-step kinds kept for the profiling hook
constexpr int kHistCols = 6;

// ---------------------------------------------------------------- state
// Which kernel does the step: the tensor-core kernel (kTcSingle / kTcSplit:
// one or two FP16 slices per operand; kTcElem: no product, epilogue only;
// kTcDelta: the second product of an FP64-accurate polishing pair, a split
// product of small matrices added to the FP64 iterate), the FP64-accurate
// SIMT kernel (kFp64 native, kDf double-float), or the FP64-accurate digit
// product on the tensor cores (kDigit).
enum Kind : int { kNone = 0, kTcSingle = 1, kTcSplit = 2, kFp64 = 3, kDf = 4, kTcElem = 5,
                  kDigit = 6, kTcDelta = 7 };
enum Phase : int { kPhaseSingle = 0, kPhaseSplit = 1, kPhaseFp64 = 2, kPhaseDone = 3 };
enum Prec : int { kPrecMixed = 0, kPrecFp64 = 1, kPrecFp32 = 2, kPrecTryFp16 = 3 };
// kMethodSp2 also runs the accelerated form (SolveState::acc_on); kMethodTrfoe
// is the truncated SP2 expansion at finite temperature.
enum Method : int { kMethodSp2 = 0, kMethodFermi = 1, kMethodTrfoe = 2 };

// Output of one tensor-core step: value = a v + b1 E1 + b2 E2 + c [i == j],
// v the product (A~ B~)_ij, E1/E2 FP32 masters of the epilogue inputs.
// kOutF64Add (with kOutF64a or kOutF64b) adds the entry of the other FP64
// buffer: Xd[1] for an output to Xd[0] and the reverse.
// kOutDiag: the diagonal form of the finite-temperature matrices, A =
// diag(d_A) + A~ with d_A an FP64 vector and A~ zero on the diagonal.  Off
// the diagonal the E terms take per-row / per-column coefficients
//     (b1 + g1r d_V1[i] + g1c d_V1[j]) E1 + (b2 + g2r d_V2[i] + g2c d_V2[j]) E2,
// and the diagonal entry, with v_ii the product's, is
//     c + a v_ii + q d_X[i] d_Y[i] + l1 d_X[i] + l2 d_Y[i],
// written to d_mat (FP64) while the small part's diagonal is stored as 0; an
// FP64 output (kOutF64a/b) writes it into the FP64 matrix instead.
enum OutFlags : int { kOutMaster = 1, kOutSlices = 2, kOutF64a = 4, kOutF64b = 8, kOutF64Add = 16,
                      kOutDiag = 32 };
struct OutSpec {
    int mat;     // target matrix slot (master and/or slices)
    int flags;   // OutFlags
    float a, b1, b2;
    float s;     // slice scale of the target
    double c;    // diagonal term, FP64 (exact for the FP64 outputs)
    // kOutDiag only: coefficient vectors of E1/E2 and the diagonal formula
    int v1, v2;                 // slots whose d vectors scale E1 / E2 (-1: none)
    float g1r, g1c, g2r, g2c;
    int dx, dy;                 // slots of the diagonal formula's d vectors (-1: none)
    double q, l1, l2;
};
struct ProdOp {
    int A, B;      // operand matrix slots (A~ and B~ slices)
    int E1, E2;    // matrix slots whose FP32 masters enter the epilogue (-1: none)
    float inv;     // v = accumulator * inv = accumulator / (s_A s_B)
    int nout;      // 1..3 outputs
    int part_out;  // output whose trace and squared Frobenius norm go to the partials
    float ra, rb, rc;  // aux partial: sum over (ra v + rb E1 + rc [i == j])^2
    int pad;
    OutSpec out[3];
};

struct SolveState {
    // problem (written by the host)
    int n;
    int prec;
    int max_iters;
    int method;
    double ne, kT, tol;
    // the tensor-core step to run next (written by the control kernel)
    ProdOp op;
    // finite temperature: beta = 1/kT, tracked chemical potential, stages
    double beta, mu_t, beta0;
    int ft_m, ft_stage, ft_sub, ft_j, ft_nj, ft_shifts, wcur, ft_phase;
    int ft_last_mat, ft_pad2;  // slot whose ||.||_F the last step's partials report
    double ns_r;      // Newton-Schulz: bound on the residual ||I - M W|| of the current W
    double ns_mmin, ns_mmax;  // bounds on the spectrum of the current M
    int ns_single;    // 1: the current Newton-Schulz pair runs single-FP16 products
    int ft_pad3;
    double sc[6];     // identity parts: A = sc I + A~ (W's in sc[kMatW0], shared by both W slots)
    double fb[6];     // bounds on ||A~||_F (slice scales are derived from them)
    float scl[6];     // slice scale s of each slot's FP16 slices (slices hold s A~)
    double ft_t, w0;  // tanh of the current shift; Newton-Schulz start
    double mu_prev;   // mu(T) of the previous tracked stage (the drift prediction)
    int mu_nconv, mu_pad;
    double tr_d0, tr_q;  // traces of D0 = (I - z)/2 and Q = (I - z^2)/4 at the end
    // spectral bounds used by the expansion (Lanczos estimate within the
    // Gershgorin interval, or Gershgorin itself) and Hp statistics
    double emin, emax, trH, hmax;
    int bad_input;
    int lz_on;            // 1: estimate the bounds with Lanczos (host sets it)
    int lz_k, lz_pad;     // Lanczos steps taken
    double gersh_lo, gersh_hi;
    double lz_a[kLanczosSteps], lz_b[kLanczosSteps + 1];
    // certificate of the estimate [lz_lo, lz_hi]: kCheckSteps logistic steps
    // X <- 4 X (I - X) from X0 on that interval; ||X||_F^2 after them (chk_F)
    // bounds how far the spectrum reaches beyond it (chk_amax, in half-widths)
    int chk_left;         // check products still to issue
    int chk;              // 1: the product issued is a check step
    double lz_lo, lz_hi, chk_F, chk_amax;
    // iterate X = c I + Y, or X = Xd[xcur] (FP64) once in the FP64 phase
    double c;
    float s_cur;        // slice scale of the current slice set
    int cur;            // current slice set (0/1)
    int xcur;           // current FP64 buffer (0/1)
    int x_fp64;         // 1: the iterate is Xd[xcur] (FP64); 0: it is c I + Y
    // which kernel runs this step (written by control)
    int kind;
    int sq;             // 1: X^2 branch, 0: 2X - X^2 branch
    float s_next;       // slice scale of the zero-temperature iterate after this step
    double c_next;
    double gamma;       // FP64-accurate step: X' = F(X) + gamma (X - X^2) (trace correction)
    // polishing pair (mixed policy): the first, FP64-accurate product also
    // writes the slices of Delta0 = X0^2 - X0 (scale pol_sD, slot Y0) and of S
    // (scale pol_sS, slot Y1); the second is X2 = X1 + pol_kappa Delta0 S
    int pol_emit, pol_pad;
    float pol_sD, pol_sS;
    double pol_kappa;
    // accelerated SP2 (A-Z-RFOE): with acc_on the unoccupied eigenvalues of X
    // lie in [acc_a, ...] = [0, acc_a] and the occupied ones in [acc_b, 1];
    // homo/lumo are the caller's estimates (host), acc_*_next the interval
    // after the product issued, acc_fold 1 when that product was folded
    int acc_on, acc_fold;
    double homo, lumo, acc_a, acc_b, acc_a_next, acc_b_next;
    // truncated SP2 at finite temperature: branch of product k in bit k
    unsigned tr_bits[kTrfoeMaxSteps / 32];
    double tr_slope;    // |dG_m/de| at the midpoint after the last product
    // convergence bookkeeping
    int iter, phase, nparts, done, status;
    int it_phase[4];
    double t1, t2, t1_prev, reltr;
    double idem_hist[3];
    double fro_hist[3];  // ||X_k^2 - X_k||_F of the inputs of the last products
    int sq_hist[2];
    // outputs
    double e_band, trace, idem_fro, mu;
    double pad[4];
    // kinds of the steps issued, in order (profiling hook)
    int nctl, nctl_pad;
    unsigned char kind_log[kKindLog];
    // per-step record written by the control kernel (read back with the state):
    // phase, branch, t1 - N_e, t1 - t2, ||X^2 - X||_F of the last product's input, RelTr
    double hist[kHistRows][kHistCols];
};

// ---------------------------------------------------------------- PTX wrappers
// x to FP32, rounded to nearest (ties to even), by integer operations on the
// FP64 encoding: GB300 runs FP64 arithmetic and FP64-to-FP32 conversions at a
// small fraction of its FP32 rate, enough to make an HBM-bound pass over FP64
// data arithmetic bound.  Values below FP32's normal range become 0, values
// above it infinity (callers pass finite data of moderate range).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
    const int fe = static_cast<int>((hi >> 20) & 0x7FFu) - 896;  // FP32 exponent field
    const unsigned sign = hi & 0x80000000u;
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
    unsigned r = (static_cast<unsigned>(fe) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;  // the 29 dropped mantissa bits
    if (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) r += 1u;  // a carry may raise the exponent
    return __uint_as_float(sign | r);
}

// Exact FP32 -> FP64 conversion by integer operations on the encodings: the
// conversion instruction runs on the FP64 pipe, which GB300 executes at 1/64
// of the FP32 rate.  Zero, subnormal, infinite and NaN inputs take the
// conversion instruction.
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return static_cast<double>(x);
    const unsigned long long r = (static_cast<unsigned long long>(b & 0x80000000u) << 32) |
                                 (static_cast<unsigned long long>(e + 896u) << 52) |
                                 (static_cast<unsigned long long>(b & 0x7FFFFFu) << 29);
    return __longlong_as_double(static_cast<long long>(r));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---- tcgen05 (5th-generation tensor core) ----
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(smem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, both K-major, FP16 inputs, FP32 accumulate.
__device__ __forceinline__ void tc_mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive FP32 columns of this warp's 32 TMEM lanes; the wait is in
// the same statement, so no use of v can be scheduled before the data lands.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float *v) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]),
          "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]),
          "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
          "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]),
          "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]),
          "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

template <uint32_t R>
__device__ __forceinline__ void setmaxnreg_inc() {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(R));
}
template <uint32_t R>
__device__ __forceinline__ void setmaxnreg_dec() {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(R));
}

// Shared-memory matrix descriptor for a K-major tile written by TMA with
// 128-byte swizzling: rows of 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *tile) {
    const uint32_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);         // start address
    d |= static_cast<uint64_t>(1u) << 16;                        // leading offset (unused, SW128 K-major)
    d |= static_cast<uint64_t>((1024u >> 4) & 0x3FFFu) << 32;   // stride offset: 8 rows x 128 B
    d |= static_cast<uint64_t>(1u) << 46;                        // descriptor version (sm_100 family)
    d |= static_cast<uint64_t>(2u) << 61;                        // swizzle mode: 128 B
    return d;
}

// The same for 64-byte swizzling: rows of 64 bytes, 8-row atoms 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw64(const void *tile) {
    const uint32_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(1u) << 16;
    d |= static_cast<uint64_t>((512u >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1u) << 46;
    d |= static_cast<uint64_t>(4u) << 61;                        // swizzle mode: 64 B
    return d;
}

// The same for 32-byte swizzling: rows of 32 bytes, 8-row atoms 256 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw32(const void *tile) {
    const uint32_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(1u) << 16;
    d |= static_cast<uint64_t>((256u >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1u) << 46;
    d |= static_cast<uint64_t>(6u) << 61;                        // swizzle mode: 32 B
    return d;
}

// Instruction descriptor: kind::f16, A and B FP16 (fmt 0) or BF16 (fmt 1),
// FP32 accumulator, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int ab_fmt) {
    return (1u << 4)                                  // D format FP32
           | (static_cast<uint32_t>(ab_fmt) << 7)     // A format
           | (static_cast<uint32_t>(ab_fmt) << 10)    // B format
           | (static_cast<uint32_t>(N >> 3) << 17)    // N / 8
           | (static_cast<uint32_t>(M >> 4) << 24);   // M / 16
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace fe
