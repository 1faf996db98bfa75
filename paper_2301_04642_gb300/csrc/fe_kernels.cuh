// Kernel entry points and the device-visible problem descriptors.
#pragma once
#include <string>

#include "fe_dev.cuh"

namespace fe {

// One symmetric n x n matrix as the tensor-core kernel sees it: FP16 slices
// (hi, lo) of s * A~ with their TMA descriptors, and optionally the FP32 master
// A~.  Zero temperature keeps (FP64 scalar) I + A~, the scalar in the solve
// state; finite temperature keeps diag(d) + A~ with d an FP64 vector
// (MmaProb::dg) and A~ zero on the diagonal, its master holding only the
// upper triangle (the epilogue reads E terms at (i, j), j >= i).
struct MatSlot {
    CUtensorMap tmA[kMaxSlices];  // box 64 (K) x 128 rows
    CUtensorMap tmB[kMaxSlices];  // box 64 (K) x 256 rows
    __half *sl[kMaxSlices];
    float *master;                // FP32 small part (null when not kept)
    long long pad;
};

// Matrix slots of a problem.  Zero temperature: kMatY0/kMatY1 are the two
// slice sets of Y (one FP32 master).  Finite temperature: z, N, M, W (two
// slice sets, one master), R.
enum MatId : int {
    kMatY0 = 0, kMatY1 = 1,
    kMatZ = 0, kMatN = 1, kMatM = 2, kMatW0 = 3, kMatW1 = 4, kMatR = 5,
    kNumMats = 6
};

// Everything the kernels need for one problem.  Lives in device global memory
// (the embedded tensor maps need 128-byte alignment); filled by the host.
struct MmaProb {
    MatSlot mats[kNumMats];
    SolveState *st;
    double *part;                    // per-tile partial slots (kPartStride doubles each)
    int n, ldy, lds, ntiles;         // ntiles: tensor-core tiles of the problem's tile width
    int ntiles64, bn;                // bn: tensor-core tile width, 128 or 256 columns
    int tc_tile0, tc_ntiles;         // this problem's range in the launch's tensor-core tile list
    float *lzv;                      // Lanczos vectors: v_prev, v, w (n FP32 each)
    float *Y;                        // FP32 master of the zero-temperature iterate
    double *Xd[2];                   // FP64 buffers (FP64 phase / finite-T output), ld ldx
    int ldx, pad0;
    const double *H;                 // Hp (device), leading dimension ldh
    long long ldh;
    // digit arrays of the FP64-accurate tensor-core product (kDigit), ld lds
    CUtensorMap dA[kDigits];         // box 32 (K) x 128 rows, 64-byte swizzle
    CUtensorMap dB[kDigits];         // box 32 (K) x 64 rows
    __half *dig[kDigits];
    int ntilesD, padD;
    double *dg[kNumMats];            // finite T: FP64 diagonals of the matrix slots (n each)
    float *dgf[kNumMats];            // their FP32 copies (the epilogue's E coefficients)
};

// One tensor-core tile: rows [I*128, I*128+128) x columns [Jp*bn, Jp*bn+bn)
// for the problem's tile width bn (256: 2Jp + 1 >= I; 128: Jp >= I).
struct TileEnt {
    int prob;
    int I;
    int Jp;
    int slot;  // partial slot index within the problem
};

// A digit-product tile uses TileEnt with Jp = J: rows [I*128, +128) x
// columns [J*64, +64), J >= 2I.

// One FP64 tile: rows [I*64, +64) x columns [J*64, +64), J >= I.
struct Tile64 {
    int prob;
    int I;
    int J;
    int slot;
};

// Split-FP16 symmetric products, Stream-K scheduled over the tiles of all
// active problems.  ws: kSkSlotFloats floats per participating CTA (partial
// sums of a split tile); cnt: 2 ints per CTA, zero between launches.
__global__ void k_sym_mma(const MmaProb *__restrict__ probs, int nprobs,
                          const TileEnt *__restrict__ tiles, int ntiles, DevCtl *ctl, float *ws, int *cnt);
constexpr size_t kSkSlotFloats = static_cast<size_t>(kTileM) * kTileN;  // 128 KiB per slot
size_t mma_smem_bytes();

struct RowInfo {
    double lo, hi, diag, maxabs;  // H_ii - r_i, H_ii + r_i, H_ii, max_j |H_ij|
};

// Gershgorin row pass: one warp per row.
__global__ void k_bounds_rows(const MmaProb *probs, int prob, RowInfo *rowinfo, int *bad);
// Deterministic reduction of the row info into the state (one block); with
// the Lanczos estimate off it also prepares X0 from the Gershgorin bounds.
__global__ void k_bounds_reduce(const MmaProb *probs, int prob, const RowInfo *rowinfo,
                                const int *bad);
// Spectral-bound estimate by kLanczosSteps Lanczos steps for the problems
// k0 .. k0 + m - 1 that have lz_on, in one cooperative launch of at most
// kLzBlocks blocks of kLzThreads (all resident at once; the host launches it
// with cudaLaunchCooperativeKernel after zeroing ctl->lz_bar): the start
// vector, then per step w = H v by every block (one warp per row, per-block
// partial dot products; v staged in `vcap` floats of dynamic shared memory
// when n <= vcap), a grid barrier, the three-term update (one block per
// problem), a grid barrier; at the end the tridiagonal is turned into the
// estimate and X0 is prepared on it.  Every barrier wait is bounded
// (kErrTimeoutGrid).  narrow < 1 shrinks the estimate about its centre by that
// factor (a test hook that forces the too-tight case).
constexpr int kLzBlocks = 304;
constexpr int kLzThreads = 512;
constexpr int kLzVcap = 24576;  // largest v staged in shared memory (96 KiB)
__global__ void k_lanczos_run(const MmaProb *probs, int k0, int m, int vcap, double narrow, DevCtl *ctl,
                              unsigned *bar);
// Certified bounds from the certificate steps (kCheckSteps products issued by
// k_control after k_lanczos_run), then the X0 preparation; one block per
// problem from k0.
__global__ void k_check_bounds(const MmaProb *probs, int k0);
// X0 = (hi I - Hp)/(hi - lo) stored as c0 I + Y0 (its slice scale from a bound
// on |Y0_ij|), or for finite temperature the parameters of z0.
__device__ __forceinline__ void setup_from_bounds(const MmaProb &pr, SolveState *st, double lo, double hi) {
    const int n = pr.n;
    st->emin = lo;
    st->emax = hi;
    const double trH = st->trH;
    double w = hi - lo;
    if (!(w > 0.0)) w = 1.0;  // Hp = a I: X0 is constant; the expansion will stall
    const double c0 = (hi - trH / n) / w;
    // |Y0_ij| <= max|Hp_ij| / w + |eps_max / w - c0|
    const double bound = st->hmax / w + fabs(hi / w - c0);
    int e;
    frexp(bound > 0.0 ? bound : 1.0, &e);  // bound < 2^e
    st->c = c0;
    st->s_cur = static_cast<float>(ldexp(1.0, 14 - e));
    st->cur = 0;
    st->xcur = 0;
    st->x_fp64 = (st->prec == kPrecFp64) ? 1 : 0;
    if (st->method == kMethodFermi) {
        // x = (beta0 / 2)(H - mu0 I) with mu0 = tr H / n and the number of
        // doublings m chosen so that |x| <= t0 = 1/4 on the bound interval;
        // the control's first five products turn x into z0 = tanh(x) (odd
        // Taylor polynomial through x^11, truncation below 5.4e-11).
        const double mu0 = trH / n;
        const double rad = fmax(fabs(lo - mu0), fabs(hi - mu0));
        const double beta = 1.0 / st->kT;
        const double t0 = 0.25;
        int m = 0;
        if (beta * rad / 2.0 > t0) m = static_cast<int>(ceil(log2(beta * rad / (2.0 * t0))));
        st->beta = beta;
        st->ft_m = m;
        st->beta0 = ldexp(beta, -m);
        st->mu_t = mu0;
        st->mu_prev = mu0;
        st->mu_nconv = 0;
        st->sc[kMatZ] = 0.0;
        int ez;
        frexp(fmax(st->beta0 * rad / 2.0, 1e-300) * 1.0001, &ez);
        st->scl[kMatZ] = static_cast<float>(ldexp(1.0, 14 - ez));
    }
}

// Zero temperature: X0 -> (c, Y0) and slices.  Finite temperature: z0.  Per-block partials.
__global__ void k_init_x0(const MmaProb *probs, int prob);
// Step control for every problem (one block per problem).
// Step bookkeeping of the graph-driven step loop (see k_control).
enum StepBits : unsigned { kStepActive = 1u, kStepTc = 2u, kStepFp64 = 4u, kStepDigit = 8u };
struct StepFlags {
    unsigned mask, count;                  // per step: OR of the problems' needs; blocks done
    unsigned n_body, n_tc, n_fp64, n_digit;  // steps run; steps that launched each family
};
// Control step: one block per problem.  With flags (inside the step graph)
// the last block to finish also sets the graph's loop and kernel switches.
// Once a kernel of the run has recorded an error in ctl (a bounded wait ran
// out), every problem ends with FE_ETIMEOUT.
__global__ void k_control(const MmaProb *probs, int nprobs, const DevCtl *ctl, StepFlags *flags,
                          cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_tc,
                          cudaGraphConditionalHandle h_fp64, cudaGraphConditionalHandle h_digit,
                          unsigned hvalid);
// FP64-accurate product + SP2 update (upper tiles, mirrored), per-tile partials.
__global__ void k_fp64_step(const MmaProb *probs, const Tile64 *tiles, int ntiles);
// D = X -> out (FP64, ld), partials of tr(H D) and tr D.
__global__ void k_finalize(const MmaProb *probs, int prob, double *D, long long ldd);
__global__ void k_finalize_reduce(const MmaProb *probs, int prob);

// FP64-accurate X^2 on the tensor cores from digit-split operands (kind kDigit).
__global__ void k_digit_mma(const MmaProb *__restrict__ probs, const TileEnt *__restrict__ tiles,
                            int ntiles, DevCtl *ctl);
size_t digit_smem_bytes();
// Digits of the current iterate for every problem whose next step is kDigit.
__global__ void k_digit_prep(const MmaProb *probs, int nprobs);

// FP32 -> FP16 slices of s*Y for a standalone product (kernel tests).
__global__ void k_make_slices(const float *Y, int n, int ldy, float s, __half *hi, __half *lo,
                              int lds);

constexpr int kInitBlocks = 608;   // 4 x 152 SMs (k_init_x0: 8 warps each, one row per warp)
constexpr int kFinBlocks = 304;
constexpr int kTile64 = 64;

// ---- products either side of the expansion in subspace iteration (k_gemm.cu)
// C = A B^T from K-major FP16 slices (hi, lo), tiles 128 x kGemmN.
constexpr int kGemmN = 192;
constexpr int kGemmThreads = 512;     // warp 0 TMA, warp 1 MMA, warps 2-3 idle, warps 4-15 drain
constexpr int kGemmDrainWarps = 12;
struct GemmArgs {
    CUtensorMap tA[kMaxSlices];       // A slices (rows_a x kdim), box 64 (K) x 128 rows
    CUtensorMap tB[kMaxSlices];       // B slices (rows_b x kdim), box 64 (K) x kGemmN rows
    double *C;                        // FP64 result, leading dimension ldc
    float *ws;                        // split mode: FP32 partial tiles, [unit][column][row]
    const unsigned long long *amax;   // [0] max|A|, [1] max|B| as FP64 bit patterns (slice scales)
    long long ldc;
    int rows_a, rows_b, kdim;
    int nsplit;                       // 0: direct C = A B^T; > 0: K in nsplit parts, k_gemm_reduce
                                      // sums them into the symmetric C (rows_a = rows_b)
    int ntiles, pad;
};
__global__ void k_gemm_split(const GemmArgs *__restrict__ args, const TileEnt *__restrict__ tiles, DevCtl *ctl);
__global__ void k_gemm_reduce(const GemmArgs *__restrict__ args, const TileEnt *__restrict__ tiles);
__global__ void k_absmax(const double *__restrict__ X, long long rows, long long cols, long long ld,
                         unsigned long long *out);
__global__ void k_split_rows(const double *__restrict__ X, long long rows, long long cols, long long ld,
                             const unsigned long long *amax, __half *hi, __half *lo, long long lds, int transpose);
size_t gemm_smem_bytes();

// Record msg as the calling thread's last error (fe_last_error_string); returns code.
int set_error_string(int code, const std::string &msg);

}  // namespace fe
