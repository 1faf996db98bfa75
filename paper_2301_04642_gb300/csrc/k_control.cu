// Per-step control on the device: no iteration needs a host synchronisation.
//
// One block per problem reduces the per-tile FP64 partials of the last
// product (fixed order), forms t1 = tr X and t2 = tr X^2 = ||X||_F^2
// (Sec. III-B), and then
//   * tests convergence with the relative trace change
//     RelTr = |t1_k - t1_{k-1}| / N_e (Sec. III-A) together with an
//     idempotency measure (the RelTr test alone leaves D^2 != D):
//       - split-FP16 phase: ||X_k^2 - X_k||_F of the product's input, which
//         the tensor-core epilogue accumulates; the phase ends when it has
//         stopped shrinking (the noise floor of the split products);
//       - FP64 phase: t1 - t2 = sum_i x_i (1 - x_i), exact enough in FP64;
//   * walks the precision schedule (Sec. III-A: cheap products while far from
//     convergence -- RelTr above 5e-4 -- accurate ones near it);
//   * picks the SP2 branch of Eq. (1): X^2 if |t2 - N_e| <= |2 t1 - t2 - N_e|
//     (the candidate whose trace is nearer N_e), else 2X - X^2;
//   * writes the coefficients the next product kernel applies.
#include <cfloat>

#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {

namespace {

// smallest power of two s with s * bound <= 2^14 (FP16 slices stay finite)
__device__ float slice_scale(double bound) {
    if (!(bound > 0.0)) bound = 1.0;
    int e;
    frexp(bound, &e);  // bound < 2^e
    return static_cast<float>(ldexp(1.0, 14 - e));
}

}  // namespace

__global__ void k_control(const MmaProb *probs, int nprobs) {
    const int p = blockIdx.x;
    if (p >= nprobs) return;
    const MmaProb &pr = probs[p];
    SolveState *st = pr.st;
    if (st->done) return;

    // number of partial slots written by the previous producer
    int nparts;
    if (st->kind == kNone) nparts = kInitBlocks;
    else if (st->kind == kFp64 || st->kind == kDf) nparts = pr.ntiles64;
    else nparts = pr.ntiles;

    __shared__ double s_a[256], s_b[256], s_c[256], s_d[256];
    const int t = threadIdx.x;
    double a = 0, b = 0, c = 0, d = 0;
    for (int k = t; k < nparts; k += blockDim.x) {
        const double *slot = pr.part + static_cast<size_t>(k) * kPartStride;
        a += slot[0];
        b += slot[1];
        c = fmax(c, slot[2]);
        d += slot[3];
    }
    s_a[t] = a; s_b[t] = b; s_c[t] = c; s_d[t] = d;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            s_a[t] += s_a[t + o];
            s_b[t] += s_b[t + o];
            s_c[t] = fmax(s_c[t], s_c[t + o]);
            s_d[t] += s_d[t + o];
        }
        __syncthreads();
    }
    if (t != 0) return;

    const double trV = s_a[0], sumsq = s_b[0], rsq = s_d[0];
    const int n = st->n;
    const double nn = static_cast<double>(n);
    const double ne = st->ne;
    const double nes = fmax(ne, 1.0);
    const int prev_kind = st->kind;

    // commit the representation produced by the previous product
    if (prev_kind == kTcSingle || prev_kind == kTcSplit) {
        st->c = st->c_next;
        st->s_cur = st->s_next;
        st->cur ^= 1;
    } else if (prev_kind == kFp64 || prev_kind == kDf) {
        st->xcur ^= 1;
        st->x_fp64 = 1;
    }
    if (prev_kind != kNone) {
        // ||X_k^2 - X_k||_F of the input of the product that just ran
        const double fro = sqrt(fmax(rsq, 0.0));
        st->idem_fro = fro;
        st->fro_hist[2] = st->fro_hist[1];
        st->fro_hist[1] = st->fro_hist[0];
        st->fro_hist[0] = fro;
    }

    if (st->bad_input) {
        st->status = -1;  // FE_EINVAL
        st->done = 1;
        st->kind = kNone;
        return;
    }

    double t1, t2;
    const double cc = st->c;
    if (st->x_fp64) {
        t1 = trV;
        t2 = sumsq;
    } else {
        t1 = n * cc + trV;
        t2 = n * cc * cc + 2.0 * cc * trV + sumsq;
    }
    const double idem = t1 - t2;
    const double reltr = (st->iter > 0) ? fabs(t1 - st->t1_prev) / nes : DBL_MAX;
    st->t1 = t1;
    st->t2 = t2;
    st->reltr = reltr;
    st->idem_hist[2] = st->idem_hist[1];
    st->idem_hist[1] = st->idem_hist[0];
    st->idem_hist[0] = idem;

    if (st->iter < kHistRows) {
        double *h = st->hist[st->iter];
        h[0] = st->phase;
        h[1] = prev_kind;
        h[2] = t1 - ne;
        h[3] = idem;
        h[4] = (prev_kind != kNone) ? st->fro_hist[0] : -1.0;
        h[5] = (st->iter > 0) ? reltr : -1.0;
    }

    // ---- precision schedule and stopping rules
    bool done = false;
    int phase = st->phase;
    if (phase == kPhaseSingle && reltr < 5e-4) phase = kPhaseSplit;  // the paper's switch point
    if (phase == kPhaseSplit && prev_kind == kTcSplit) {
        // The split products carry ~22 bits and the FP32 master 24, so the
        // eigenvalue deviations cannot be pushed much below ~2^-22: stop at
        // the first ||X^2 - X||_F at that level (2^-20 sqrt(N_e) leaves a
        // margin), or as soon as it stops shrinking.
        const double f0 = st->fro_hist[0], f2 = st->fro_hist[2];
        const double floor_level = 9.5367431640625e-07 * sqrt(fmax(ne, 1.0));  // 2^-20
        const bool floor = st->iter >= 4 &&
                           (f0 <= floor_level || (f0 <= 1e-4 * sqrt(nn) && f0 >= 0.5 * f2));
        if (floor) {
            if (st->prec == kPrecFp32) done = true;
            else phase = kPhaseFp64;
        }
    } else if (phase == kPhaseFp64 && (prev_kind == kFp64 || prev_kind == kDf)) {
        const int nfp64 = st->it_phase[kPhaseFp64];
        const bool idem_ok = fabs(idem) <= 2e-10 ||
                             (fabs(idem) >= 0.5 * fabs(st->idem_hist[2]) && fabs(idem) <= 1e-6);
        if (st->prec == kPrecFp64) {
            if (reltr <= st->tol && idem_ok) done = true;
        } else {
            // Polishing products come in pairs of opposite branches, the second
            // one carrying the exact trace correction (below): after a pair the
            // deviations are O(dx^2) on both sides and tr X = N_e to rounding.
            // fro_hist[0] = ||X^2 - X||_F of the pair's second input; the
            // output's deviations are about its square
            (void)idem_ok;
            const double f0 = st->fro_hist[0];
            if (nfp64 >= 2 && (nfp64 & 1) == 0 &&
                ((f0 * f0 <= 5e-9 && fabs(idem) <= 1e-8) || nfp64 >= 6))
                done = true;
        }
    }
    if (!done && st->iter >= st->max_iters) {
        st->status = -3;  // FE_ENOTCONV
        done = true;
    }
    if (done) {
        st->done = 1;
        st->phase = kPhaseDone;
        st->kind = kNone;
        return;
    }

    // ---- SP2 branch (Eq. (1)) and the instruction for the next product
    int sq = fabs(t2 - ne) <= fabs(2.0 * t1 - t2 - ne);
    // Polishing (mixed schedules): the second product of each pair takes the
    // other branch, so a pair maps x -> 1 - O(dx^2) near 1 and O(dx^2) near
    // 0 whichever side the trace rule favoured first.
    st->gamma = 0.0;
    if (phase == kPhaseFp64 && st->prec != kPrecFp64 && (st->it_phase[kPhaseFp64] & 1) == 1) {
        sq = !st->sq;
        // Exact trace: the branch output F(X) has trace t2 (X^2) or 2 t1 - t2
        // (2X - X^2), known now from the FP64 partials of X; adding
        // gamma (X - X^2), whose trace is t1 - t2, lands tr X' on N_e.
        // The correction moves eigenvalue x by gamma x (1 - x); |x (1 - x)| of
        // this iterate is at most ~2 ||X_prev^2 - X_prev||_F (one side of the
        // first product of the pair doubled).  Apply it only when a trace error
        // remains and the largest move stays within a few times that error,
        // i.e. when the x (1 - x) do not cancel in their sum.
        const double trF = sq ? t2 : 2.0 * t1 - t2;
        const double dtr = ne - trF;
        const double dev = t1 - t2;
        if (fabs(dtr) > 5e-11 && fabs(dev) > 1e-14 * nes) {
            const double g = dtr / dev;
            const double max_move = fabs(g) * 2.0 * st->fro_hist[0];
            if (fabs(g) <= 0.5 && max_move <= fmax(4.0 * fabs(dtr), 1e-10)) st->gamma = g;
        }
    }
    st->sq = sq;
    st->phase = phase;
    if (phase == kPhaseFp64) {
        st->kind = (st->prec == kPrecFp64) ? kFp64 : kDf;
    } else {
        st->kind = (phase == kPhaseSingle) ? kTcSingle : kTcSplit;
        const double alpha = sq ? 2.0 * cc : 2.0 - 2.0 * cc;
        const double cn = sq ? cc * cc : 2.0 * cc - cc * cc;
        st->alpha = static_cast<float>(alpha);
        st->sigma = sq ? 1.0f : -1.0f;
        st->c_next = cn;
        st->r1 = static_cast<float>(2.0 * cc - 1.0);
        st->r0 = static_cast<float>(cc * cc - cc);
        const double s = st->s_cur;
        st->inv_s2 = static_cast<float>(1.0 / (s * s));
        // entries of Y' = X' - c' I are bounded by its spectral radius:
        // spec(X') in [0, 1] gives max(c', 1 - c'); also ||alpha Y + sigma Y^2||_F
        const double fro = sqrt(fmax(sumsq, 0.0));
        const double bound = fmin(fmax(cn, 1.0 - cn) + 1e-3, fabs(alpha) * fro + fro * fro);
        st->s_next = slice_scale(bound * 1.0001);
    }
    st->t1_prev = t1;
    st->it_phase[phase] += 1;
    st->iter += 1;
}

}  // namespace fe
