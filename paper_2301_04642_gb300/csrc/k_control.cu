// Per-step control on the device: no iteration needs a host synchronisation.
// One block per problem reduces the per-tile FP64 partials of the last step
// (fixed order) and writes the next step into the solve state.
//
// Zero temperature (SP2, Sec. II-B1 Eq. (1)):
//   * t1 = tr X, t2 = tr X^2 = ||X||_F^2 (Sec. III-B);
//   * convergence: relative trace change RelTr = |t1_k - t1_{k-1}| / N_e
//     (Sec. III-A) together with an idempotency measure (the RelTr test alone
//     leaves D^2 != D): in the split-FP16 phase ||X_k^2 - X_k||_F, which the
//     tensor-core epilogue accumulates; in the FP64-accurate phase
//     t1 - t2 = sum_i x_i (1 - x_i);
//   * precision schedule (Sec. III-A: cheap products while far from
//     convergence, accurate ones near it);
//   * branch: X^2 if |t2 - N_e| <= |2 t1 - t2 - N_e| (the candidate whose trace
//     is nearer N_e), else 2X - X^2.
//
// Finite temperature (Sec. II-A Fermi-Dirac target, recursive expansion of
// Sec. II-B3): z = I - 2D = tanh(beta (H - mu)/2).  Starting from
// z0 = tanh((beta0/2)(H - mu0 I)) at beta0 = beta / 2^m (the paper's
// expansion starts from the linear term; here six products evaluate a
// Taylor polynomial of tanh instead, see control_fermi_start), every stage
// doubles beta with the double-angle identity of tanh, folding in a shift of
// mu (logit shift b, t = tanh b) chosen by a Newton step so that tr D tracks
// N_e at every temperature:
//   z' = (z - t)(I - t z)^{-1}  and  z'' = 2 z' (I + z'^2)^{-1}
//   => z'' = N M^{-1},  N = 2 ((1 + t^2) z - t (I + z^2)),
//                       M = (1 + t^2)(I + z^2) - 4 t z.
// M^{-1} comes from Newton-Schulz, W <- W (2 I - M W), started at the
// scalar w0 = 2 / (m_min + m_max) from bounds of M's spectrum over
// z in [-rho, rho], rho = tanh(beta_k R / 2) with R the Gershgorin radius
// around mu: early stages (small z, M close to I) need few or no steps.
// After the last stage up to three shift-only steps N = z - t I, M = I - t z
// bring tr D near N_e, and a last product writes D0 = (I - z)/2 and
// Q = (I - z^2)/4 = D0 - D0^2 in FP64; the output kernel forms
// D = D0 + gamma Q with gamma fixed so that tr D = N_e exactly (a first-order
// shift of mu, since dD/dmu = beta D (I - D)).
// All matrices are kept as diag(FP64 vector) + (FP32 small part, zero on the
// diagonal); every product is a split-FP16 tensor-core product of the small
// parts (see the diagonal form below).
#include <cfloat>

#include "fe_dev.cuh"
#include "fe_kernels.cuh"

namespace fe {

namespace {

// smallest power of two s with s * bound <= 2^14 (FP16 slices stay finite)
__device__ float slice_scale(double bound) {
    if (!(bound > 0.0)) bound = 1.0;
    int e;
    frexp(bound * 1.0001, &e);  // bound < 2^e
    return static_cast<float>(ldexp(1.0, 14 - e));
}

__device__ void set_out(OutSpec &o, int mat, int flags, double a, double b1, double b2, double c,
                        double bound) {
    o.mat = mat;
    o.flags = flags;
    o.a = static_cast<float>(a);
    o.b1 = static_cast<float>(b1);
    o.b2 = static_cast<float>(b2);
    o.c = c;
    o.s = slice_scale(bound);
    o.v1 = o.v2 = o.dx = o.dy = -1;
    o.g1r = o.g1c = o.g2r = o.g2c = 0.0f;
    o.q = o.l1 = o.l2 = 0.0;
}

__device__ void begin_op(ProdOp &op, int A, int B, int E1, int E2, double inv) {
    op.A = A;
    op.B = B;
    op.E1 = E1;
    op.E2 = E2;
    op.inv = static_cast<float>(inv);
    op.nout = 0;
    op.part_out = 0;
    op.ra = op.rb = op.rc = 0.0f;
}

// ------------------------------------------------------ bound certificate
// The kCheckSteps logistic steps X <- 4 X (I - X) that certify the spectral-
// bound estimate (the derivation is with k_check_bounds).  X0 was prepared on
// the estimate in the zero-temperature form for either method; the products
// use the split-FP16 kernel (the FP64 kernel for FP64-only problems).  After
// the last one, chk_amax bounds |a| over the spectrum, a in half-widths of
// the estimate about its centre.
__device__ void control_check(SolveState *st, double trV, double sumsq) {
    const int n = st->n;
    const int prev = st->kind;
    if (prev == kTcSplit) {
        st->c = st->c_next;
        st->s_cur = st->s_next;
        st->cur ^= 1;
    } else if (prev == kFp64) {
        st->xcur ^= 1;
    }
    const double cc = st->c;
    const double f2 = st->x_fp64 ? sumsq : n * cc * cc + 2.0 * cc * trV + sumsq;  // ||X||_F^2
    if (st->chk_left == 0) {
        // |T_8(a)| = |1 - 2 x_3| <= 1 + 2 ||X_3||_F for every eigenvalue; the
        // allowance (a quarter of ||X_3||_F, plus 1) covers the products'
        // rounding: FP16 slices of ~22 bits and FP32 sums, a relative error of
        // order 1e-5 after three products even where the rounding is one-sided
        const double f = sqrt(fmax(f2, 0.0));
        const double t = 1.0 + 2.0 * (1.25 * f + 1.0);
        st->chk_F = f2;
        st->chk_amax = cosh(acosh(t) / static_cast<double>(1 << kCheckSteps));
        st->chk = 0;
        st->kind = kNone;
        return;
    }
    st->chk = 1;
    st->chk_left -= 1;
    if (st->x_fp64) {
        st->kind = kFp64;
        return;
    }
    // X = c I + Y:  4X - 4X^2 -> c' = 4c - 4c^2, Y' = (4 - 8c) Y - 4 Y^2, with
    // ||Y'||_F <= |4 - 8c| ||Y||_F + 4 ||Y||_F^2 (no [0, 1] assumption here)
    const double alpha = 4.0 - 8.0 * cc;
    const double fro = sqrt(fmax(sumsq, 0.0));
    const double bound = fabs(alpha) * fro + 4.0 * fro * fro;
    st->kind = kTcSplit;
    st->c_next = 4.0 * cc - 4.0 * cc * cc;
    ProdOp &op = st->op;
    const int cur = st->cur;
    const double s = st->s_cur;
    begin_op(op, cur, cur, cur, -1, 1.0 / (s * s));
    op.nout = 1;
    // the last step's matrix is not used again, only its trace and Frobenius
    // norm (X0 is prepared afresh on the certified bounds): no stores
    const int fl = (st->chk_left == 0) ? 0 : (kOutMaster | kOutSlices);
    set_out(op.out[0], cur ^ 1, fl, -4.0, alpha, 0.0, 0.0, bound);
    st->s_next = op.out[0].s;
}

// ------------------------------------------------------------------ SP2 step
__device__ void control_sp2(SolveState *st, double trV, double sumsq, double rsq) {
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
    } else if (prev_kind == kFp64 || prev_kind == kDf || prev_kind == kDigit || prev_kind == kTcDelta) {
        st->xcur ^= 1;
        st->x_fp64 = 1;
    }
    st->pol_emit = 0;
    if (st->acc_fold) {
        st->acc_a = st->acc_a_next;
        st->acc_b = st->acc_b_next;
    }
    if (st->acc_on && st->iter == 0) {
        // A-Z-RFOE (Sec. II-B2): with X0 = (eps_max I - H)/w the estimates
        // put the unoccupied eigenvalues in [0, a] and the occupied ones in
        // [b, 1]; estimates that do not bracket a gap inside the bounds give
        // no information (plain SP2)
        const double w = st->emax - st->emin;
        const double a = (st->emax - st->lumo) / w, b = (st->emax - st->homo) / w;
        if (w > 0.0 && a >= 0.0 && b <= 1.0 && a < b) {
            st->acc_a = a;
            st->acc_b = b;
        } else {
            st->acc_on = 0;
        }
    }
    if (prev_kind != kNone) {
        // ||X_k^2 - X_k||_F of the input of the product that just ran
        const double fro = sqrt(fmax(rsq, 0.0));
        st->idem_fro = fro;
        st->fro_hist[2] = st->fro_hist[1];
        st->fro_hist[1] = st->fro_hist[0];
        st->fro_hist[0] = fro;
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
    // With every eigenvalue of X in [0, 1], t2 <= t1 and 0 <= t1 <= n.  An
    // eigenvalue outside the spectral-bound estimate can end on the wrong side
    // only after leaving [-0.37, 1.37], where x (x - 1) > 0.5: stop, and the
    // host solves again from the Gershgorin bounds.
    if (!(t2 <= t1 + 0.5) || t1 < -0.5 || t1 > nn + 0.5) {
        st->status = st->lz_on ? kStatusEscaped : -3;  // -3: FE_ENOTCONV
        done = true;
    }
    if (!done && st->acc_on && st->acc_fold) {
        // The folds keep N_e eigenvalues in [b, 1] and n - N_e in [0, a] only
        // when the HOMO/LUMO estimates lie inside the gap.  Then
        //   N_e b <= tr X <= N_e + (n - N_e) a,
        //   tr X - tr X^2 = sum x (1 - x) <= (n - N_e) a + N_e (1 - b);
        // a state on the wrong side, or one left between a and b, breaks one
        // of these by a whole state once a and 1 - b are small.  A violation
        // by more than 1/2 ends this attempt; the host runs plain SP2.
        const double a = st->acc_a, b = st->acc_b;
        const double spread = (nn - ne) * a + ne * (1.0 - b);
        if (t1 < ne * b - 0.5 || t1 > ne + (nn - ne) * a + 0.5 || idem > spread + 0.5) {
            st->status = kStatusAccelFailed;
            done = true;
        }
    }
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
    } else if (phase == kPhaseFp64 &&
               (prev_kind == kFp64 || prev_kind == kDf || prev_kind == kDigit || prev_kind == kTcDelta)) {
        const int nfp64 = st->it_phase[kPhaseFp64];
        if (st->prec == kPrecFp64) {
            const bool idem_ok = fabs(idem) <= 2e-10 ||
                                 (fabs(idem) >= 0.5 * fabs(st->idem_hist[2]) && fabs(idem) <= 1e-6);
            if (reltr <= st->tol && idem_ok) done = true;
        } else {
            // Polishing products come in pairs of opposite branches, the second
            // carrying the exact trace correction (below); after a pair the
            // deviations are about the square of fro_hist[0] = ||X^2 - X||_F of
            // the pair's second input.  The trace must also have landed: when
            // the correction was not admissible (deviations of both signs
            // cancel in tr(X - X^2)), further products square what is left.
            // After a pair every eigenvalue's x (1 - x) is >= 0 (squared
            // deviations), so t1 - t2 = sum x (1 - x) bounds ||X^2 - X||_F;
            // from then on a single product may end the phase (the SP2 rule
            // picks the branch that squares the side holding the trace
            // error, e.g. one slowly converging eigenvalue next to the gap).
            // t1 and t2 are both about N_e and carry the rounding of their
            // FP64 sums (measured: 11 ulp(N_e) below zero at n = 16040), so
            // the sign test on their difference allows N_e 2^-46 (64 to 128
            // ulp of N_e).
            const double f0 = st->fro_hist[0];
            const double idem_floor = -fmax(1e-12, ldexp(fmax(ne, 1.0), -46));
            const bool idem_small = idem >= idem_floor && idem <= 5e-9;
            const bool trace_ok = fabs(t1 - ne) <= 5e-10;
            const bool pair_ok = (nfp64 & 1) == 0 ? f0 * f0 <= 5e-9 : true;
            if (nfp64 >= 2 && idem_small && trace_ok && pair_ok) {
                done = true;
            } else if (nfp64 >= 6) {
                // three pairs did not reach the trace and idempotency targets
                // (a HOMO/LUMO gap too small to resolve, or a degenerate
                // Fermi level split by N_e): D is not the projector
                st->status = -3;  // FE_ENOTCONV
                done = true;
            }
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
    if (st->acc_on && phase != kPhaseFp64 && fmax(st->acc_a, 1.0 - st->acc_b) >= 1e-3) {
        // A-Z-RFOE: the bounds say where the gap is; the branch moves it
        // toward the middle of [0, 1] (the trace rule takes over once the
        // folds are negligible)
        sq = st->acc_a + st->acc_b > 1.0;
    }
    st->gamma = 0.0;
    if (phase == kPhaseFp64 && st->prec != kPrecFp64 && (st->it_phase[kPhaseFp64] & 1) == 1) {
        // Polishing: the second product of each pair takes the other branch,
        // so a pair maps x -> 1 - O(dx^2) near 1 and O(dx^2) near 0.
        sq = !st->sq;
        // Exact trace: the branch output F(X) has trace t2 (X^2) or 2 t1 - t2
        // (2X - X^2); adding gamma (X - X^2), of trace t1 - t2, lands tr X' on
        // N_e.  gamma moves eigenvalue x by gamma x (1 - x); this input's
        // deviations are first order (one side of the pair is not squared
        // yet), so the move is at most |gamma| 2 ||X_prev^2 - X_prev||_F in
        // Frobenius norm.  It is applied only while that stays within the
        // idempotency budget (2e-9); otherwise the next product's branch
        // squares what is left and takes the trace with it.
        const double trF = sq ? t2 : 2.0 * t1 - t2;
        const double dtr = ne - trF;
        const double dev = t1 - t2;
        if (fabs(dtr) > 5e-11 && fabs(dev) > 1e-14 * nes) {
            const double g = dtr / dev;
            const double max_move = fabs(g) * 2.0 * st->fro_hist[0];
            if (fabs(g) <= 0.5 && max_move <= 2e-9) st->gamma = g;
        }
    }
    st->sq = sq;
    st->phase = phase;
    st->acc_fold = 0;
    if (phase == kPhaseFp64) {
        st->acc_on = 0;  // the FP64-accurate steps are plain SP2 (a and 1 - b are ~0 by now)
        if (st->prec == kPrecFp64) {
            st->kind = kFp64;
        } else if ((st->it_phase[kPhaseFp64] & 1) == 0) {
            // First product of a polishing pair: FP64-accurate, X1 = F_A(X0).
            // Its epilogue also writes the slices of Delta0 = X0^2 - X0 and of
            // S = 2 X0 + Delta0 (X^2 branch) or 2I - 2 X0 + Delta0.  Slice
            // scales from bounds on the spectral norms (entries are below
            // them): |S| <= 2 max|x| + ||Delta0|| < 4; X0 = F(X_in) doubles
            // the deviations of X_in on one side (||.||_F <= fro_hist[0]) and
            // squares them on the other, plus the rounding of the product
            // that made X0: at most 2^-19 n for a split product (entries of
            // Y^2 within 2^-20 of exact, FP32 master), 2^-40 n once FP64.
            st->kind = kDigit;
            st->pol_emit = 1;
            const double f = st->fro_hist[0];
            const double bD = 4.0 * f + f * f + ldexp(nn, st->x_fp64 ? -40 : -19);
            st->pol_sD = slice_scale(bD);
            st->pol_sS = slice_scale(4.0);
        } else {
            // Second product of the pair, with Delta0 and X0 commuting:
            //   X1 = X0^2 = X0 + Delta0     ->  Delta1 = X1^2 - X1 = Delta0 (2 X0 + Delta0)
            //   X1 = 2 X0 - X0^2 = X0 - Delta0 -> Delta1 = Delta0 (2I - 2 X0 + Delta0)
            // and F_B(X1) + gamma (X1 - X1^2) = X1 + kappa Delta1 with
            // kappa = 1 - gamma (X^2 branch) or -1 - gamma (2X - X^2).
            // Delta0 is small, so the split-FP16 product gives Delta1 to
            // ~2^-21 of |Delta0| |S|, an absolute error far below the FP64
            // iterate's tolerance; X1 + kappa Delta1 is formed in FP64.
            st->kind = kTcDelta;
            st->pol_kappa = sq ? 1.0 - st->gamma : -1.0 - st->gamma;
            ProdOp &op = st->op;
            begin_op(op, kMatY0, kMatY1, -1, -1, 1.0 / (static_cast<double>(st->pol_sD) * st->pol_sS));
            op.nout = 1;
            set_out(op.out[0], kMatY0, kOutF64Add | ((st->xcur ^ 1) == 0 ? kOutF64a : kOutF64b),
                    st->pol_kappa, 0.0, 0.0, 0.0, 1.0);
            op.part_out = 0;
            op.ra = 1.0f;  // ||Delta1||_F^2 = ||X1^2 - X1||_F^2 of this product's input
        }
    } else {
        st->kind = (phase == kPhaseSingle) ? kTcSingle : kTcSplit;
        // The step's polynomial, folded over the interval that has to shrink
        // when A-Z-RFOE is on (fold point sf; sf = 0 is the SP2 step):
        //   X^2 branch:      X' = r (X - sf I)^2,             sf = a / 2
        //   2X - X^2 branch: X' = r (2 (1 - sf) X - X^2),    sf = (1 - b) / 2
        // with r = 1 / (1 - sf)^2.  With X = c I + Y:
        //   X^2:      c' = r (c - sf)^2,            Y' = r (2 (c - sf) Y + Y^2)
        //   2X - X^2: c' = r (2 (1 - sf) c - c^2),  Y' = r ((2 (1 - sf) - 2c) Y - Y^2)
        double sf = 0.0;
        if (st->acc_on) {
            sf = sq ? 0.5 * st->acc_a : 0.5 * (1.0 - st->acc_b);
            // a product's rounding error enters X' multiplied by r and turns
            // the occupied subspace by that error over the gap b - a: while
            // the gap is narrow the fold is capped at sf <= 1/4 (r <= 16/9)
            if (st->acc_b - st->acc_a < 1e-2 && sf > 0.25) sf = 0.25;
            const double rr = 1.0 / ((1.0 - sf) * (1.0 - sf));
            const double a = st->acc_a, b = st->acc_b;
            st->acc_a_next = sq ? rr * (a - sf) * (a - sf) : rr * (2.0 * (1.0 - sf) * a - a * a);
            st->acc_b_next = sq ? rr * (b - sf) * (b - sf) : rr * (2.0 * (1.0 - sf) * b - b * b);
            st->acc_fold = 1;
        }
        const double r = 1.0 / ((1.0 - sf) * (1.0 - sf));
        const double alpha = sq ? 2.0 * (cc - sf) : 2.0 * (1.0 - sf) - 2.0 * cc;
        const double cn = sq ? r * ((cc - sf) * (cc - sf)) : r * (2.0 * (1.0 - sf) * cc - cc * cc);
        st->c_next = cn;
        // entries of Y' = X' - c' I are bounded by its spectral radius:
        // spec(X') in [0, 1] gives max(c', 1 - c'); also r ||alpha Y + sigma Y^2||_F
        const double fro = sqrt(fmax(sumsq, 0.0));
        const double bound = fmin(fmax(cn, 1.0 - cn) + 1e-3, r * (fabs(alpha) * fro + fro * fro));
        const int cur = st->cur;
        ProdOp &op = st->op;
        const double s = st->s_cur;
        begin_op(op, cur, cur, cur, -1, 1.0 / (s * s));
        op.nout = 1;
        set_out(op.out[0], cur ^ 1, kOutMaster | kOutSlices, sq ? r : -r, r * alpha, 0.0, 0.0, bound);
        st->s_next = op.out[0].s;
        // ||X^2 - X||: X^2 - X = Y^2 + (2c - 1) Y + (c^2 - c) I
        op.ra = 1.0f;
        op.rb = static_cast<float>(2.0 * cc - 1.0);
        op.rc = static_cast<float>(cc * cc - cc);
    }
    st->t1_prev = t1;
    st->it_phase[phase] += 1;
    st->iter += 1;
}

// ------------------------------------------------- truncated SP2 at finite T
// The paper's T-RFOE (Sec. II-B3, Eq. (2)): D = G_m(X0), the SP2 recursion
// with the trace rule stopped after m products, X0 from the Gershgorin
// bounds.  m is read as the first step whose step function is as steep at
// its midpoint (G_m = 1/2) as Fermi-Dirac at mu: |dG_m/de| >= beta / 4.
// With u_m = 1/2 and u_k = F_k^{-1}(u_{k+1}) (sqrt(y) after X^2,
// 1 - sqrt(1 - y) after 2X - X^2), |dG_m/de| = (1/w) prod F_k'(u_k),
// F' = 2u or 2 - 2u, and the midpoint energy is eps_max - w u_0.
__device__ double trfoe_slope(const SolveState *st, int m, double w, double *mid) {
    double u = 0.5, d = 1.0;
    for (int k = m - 1; k >= 0; --k) {
        const bool sq = (st->tr_bits[k >> 5] >> (k & 31)) & 1u;
        u = sq ? sqrt(u) : 1.0 - sqrt(1.0 - u);
        d *= sq ? 2.0 * u : 2.0 - 2.0 * u;
    }
    *mid = u;
    return d / w;
}

__device__ void control_trfoe(SolveState *st, double trV, double sumsq) {
    const int n = st->n;
    const double ne = st->ne;
    const double nes = fmax(ne, 1.0);
    const int prev_kind = st->kind;
    if (prev_kind == kTcSingle || prev_kind == kTcSplit) {
        st->c = st->c_next;
        st->s_cur = st->s_next;
        st->cur ^= 1;
    } else if (prev_kind == kFp64 || prev_kind == kDf || prev_kind == kDigit) {
        st->xcur ^= 1;
        st->x_fp64 = 1;
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
    const double reltr = (st->iter > 0) ? fabs(t1 - st->t1_prev) / nes : DBL_MAX;
    st->t1 = t1;
    st->t2 = t2;
    st->reltr = reltr;
    const int m = st->iter;
    const double w = st->emax - st->emin;
    double mid;
    const double slope = trfoe_slope(st, m, w > 0.0 ? w : 1.0, &mid);
    st->tr_slope = slope;
    if (st->iter < kHistRows) {
        double *h = st->hist[st->iter];
        h[0] = st->phase;
        h[1] = prev_kind;
        h[2] = t1 - ne;
        h[3] = t1 - t2;
        h[4] = slope;
        h[5] = (st->iter > 0) ? reltr : -1.0;
    }
    if (slope >= 0.25 * st->beta) {
        st->mu = st->emax - w * mid;
        st->done = 1;
        st->phase = kPhaseDone;
        st->kind = kNone;
        return;
    }
    const int cap = st->max_iters < kTrfoeMaxSteps ? st->max_iters : kTrfoeMaxSteps;
    if (m >= cap) {
        st->status = -3;  // FE_ENOTCONV
        st->done = 1;
        st->phase = kPhaseDone;
        st->kind = kNone;
        return;
    }
    // precision: split FP16 products until RelTr < 5e-4 (the paper's switch
    // point), then FP64-accurate ones; FP32 keeps the split products
    int phase = st->phase;
    if (phase == kPhaseSplit && st->prec == kPrecMixed && m > 0 && reltr < 5e-4) phase = kPhaseFp64;
    const int sq = fabs(t2 - ne) <= fabs(2.0 * t1 - t2 - ne);
    if (sq) st->tr_bits[m >> 5] |= 1u << (m & 31);
    else st->tr_bits[m >> 5] &= ~(1u << (m & 31));
    st->sq = sq;
    st->gamma = 0.0;
    st->phase = phase;
    if (phase == kPhaseFp64) {
        st->kind = kDigit;  // FP64-accurate tensor-core products (FE_PREC_FP64 from the start)
    } else {
        st->kind = kTcSplit;
        const double alpha = sq ? 2.0 * cc : 2.0 - 2.0 * cc;
        const double cn = sq ? cc * cc : 2.0 * cc - cc * cc;
        st->c_next = cn;
        const double fro = sqrt(fmax(sumsq, 0.0));
        const double bound = fmin(fmax(cn, 1.0 - cn) + 1e-3, fabs(alpha) * fro + fro * fro);
        const int cur = st->cur;
        ProdOp &op = st->op;
        const double s = st->s_cur;
        begin_op(op, cur, cur, cur, -1, 1.0 / (s * s));
        op.nout = 1;
        set_out(op.out[0], cur ^ 1, kOutMaster | kOutSlices, sq ? 1.0 : -1.0, alpha, 0.0, 0.0, bound);
        st->s_next = op.out[0].s;
        op.ra = 1.0f;
        op.rb = static_cast<float>(2.0 * cc - 1.0);
        op.rc = static_cast<float>(cc * cc - cc);
    }
    st->t1_prev = t1;
    st->it_phase[phase] += 1;
    st->iter += 1;
}

// ------------------------------------------------------------------ finite T
// ft_sub names the step that was issued last; kFtStart is the state after X0.
enum FtSub : int { kFtStart = 0, kFtSquare = 1, kFtShiftElem = 2, kFtMW = 3, kFtWR = 4, kFtNW = 5,
                   kFtFinal = 6, kFtPoly1 = 7, kFtPoly2 = 8, kFtPoly3 = 9, kFtPoly4 = 10, kFtPoly5 = 11,
                   kFtPoly6 = 12 };

// Finite-temperature matrices are kept in the diagonal form A = diag(d_A) +
// A~ (d_A FP64, A~ FP32 master + FP16 slices, zero on the diagonal; the
// kOutDiag epilogue).  With both operands in that form
//     (A B)_ij = d_A[i] B~_ij + A~_ij d_B[j] + (A~ B~)_ij   (i != j),
//     (A B)_ii = d_A[i] d_B[i] + (A~ B~)_ii,
// so every output is the product v = A~ B~ plus E terms with per-row or
// per-column coefficients, and its diagonal is formed in FP64.  Why: near
// the Fermi level the Fermi function's slope beta/4 amplifies an absolute
// error of the logit, and with (scalar) I + A~ the diagonal entries of A~
// are O(1) (A's diagonal minus its mean), so their FP32/FP16 rounding is an
// absolute 2^-23..2^-24 on every eigenvalue whose eigenvector is localised
// (Hp close to diagonal, as late in a self-consistent cycle).  In a CPU
// emulation with the kernels' slicing (n = 800, kT = 1.2 mHa, reflector Q)
// ||D - D_ref||_F / sqrt(N_e) was 9.5e-7 in the scalar form and 3.6e-8 in
// the diagonal form (1.5e-7 and 8.7e-8 for a Haar Q).
//
// Slice scales come from spectral bounds of the full matrices: entries of
// the off-diagonal part A~ are below ||A~||_2 <= 2 ||A||_2.
__device__ float ft_scale(double spec) { return slice_scale(2.5 * spec + 1e-6); }

// E-term coefficients and the diagonal formula of a diagonal-form output
__device__ void set_e(OutSpec &o, int v1, double b1, double g1r, double g1c, int v2, double b2, double g2r,
                      double g2c) {
    o.flags |= kOutDiag;
    o.v1 = v1;
    o.b1 = static_cast<float>(b1);
    o.g1r = static_cast<float>(g1r);
    o.g1c = static_cast<float>(g1c);
    o.v2 = v2;
    o.b2 = static_cast<float>(b2);
    o.g2r = static_cast<float>(g2r);
    o.g2c = static_cast<float>(g2c);
}
__device__ void set_d(OutSpec &o, double c, int dx, int dy, double q, double l1, double l2) {
    o.flags |= kOutDiag;
    o.c = c;
    o.dx = dx;
    o.dy = dy;
    o.q = q;
    o.l1 = l1;
    o.l2 = l2;
}
// output = a v + E terms; diagonal c + a v_ii + q d_X d_Y + l1 d_X + l2 d_Y
__device__ void out_d(OutSpec &o, int mat, int flags, double a, double spec) {
    o.mat = mat;
    o.flags = flags | kOutDiag;
    o.a = static_cast<float>(a);
    o.b1 = o.b2 = 0.0f;
    o.g1r = o.g1c = o.g2r = o.g2c = 0.0f;
    o.v1 = o.v2 = o.dx = o.dy = -1;
    o.c = o.q = o.l1 = o.l2 = 0.0;
    o.s = ft_scale(spec);
}
// the product of two diagonal-form matrices A B (commuting, so symmetric):
// E1 = B~ scaled by d_A per row, E2 = A~ scaled by d_B per column
__device__ void prod_terms(OutSpec &o, int A, int B, double a) {
    set_e(o, A, 0.0, a, 0.0, B, 0.0, 0.0, a);
    set_d(o, 0.0, A, B, a, 0.0, 0.0);
}

// The start z0 = tanh(x), x = (beta0/2)(H - mu0 I) with ||x||_2 <= 1/4 on the
// bound interval, from the odd Taylor polynomial of tanh through x^11 in
// Horner form in y = x^2:
//   tanh x = x P,  P = c0 + y T2,  T2 = c1 + y T3,  T3 = c2 + y T4,
//   T4 = c3 + y T5,  T5 = c4 + c5 y
// (the next term, 21844/6081075 x^13, is below 5.4e-11 at |x| = 1/4).  Six
// split-FP16 products replace the eight doublings from |x| <= 1e-3 to 1/4.
//   1: Y = x x -> M, T5 -> N, copy of x -> R     2: T4 = c3 + Y T5 -> W0
//   3: T3 = c2 + Y T4 -> N     4: T2 = c1 + Y T3 -> W0     5: P = c0 + Y T2 -> N
//   6: z0 = x P -> Z
__device__ double tanh_coef(int k) {
    switch (k) {
        case 0: return 1.0;
        case 1: return -1.0 / 3.0;
        case 2: return 2.0 / 15.0;
        case 3: return -17.0 / 315.0;
        case 4: return 62.0 / 2835.0;
        default: return -1382.0 / 155925.0;
    }
}

__device__ void control_fermi_start(SolveState *st, int sub) {
    float *scl = st->scl;
    ProdOp &op = st->op;
    const int Z = kMatZ, N = kMatN, M = kMatM, W0 = kMatW0, X = kMatR;
    // r bounds ||x||_2 (bound interval about mu0)
    const double r = 0.5 * st->beta0 * fmax(fabs(st->emax - st->mu_t), fabs(st->emin - st->mu_t));
    const double r2 = r * r;
    // spectral bounds of T5, T4, T3, T2, P over y in [0, r^2]
    double tb[6];
    tb[5] = fabs(tanh_coef(4)) + fabs(tanh_coef(5)) * r2;
    for (int k = 4; k >= 1; --k) tb[k] = fabs(tanh_coef(k - 1)) + r2 * tb[k + 1];
    st->kind = kTcSplit;
    op.part_out = 0;
    auto horner = [&](int T, int out, int k, double spec) {
        // out = c_k I + Y T with Y in M: E1 = T~ (row d_Y), E2 = Y~ (column d_T)
        begin_op(op, M, T, T, M, 1.0 / (static_cast<double>(scl[M]) * scl[T]));
        op.nout = 1;
        out_d(op.out[0], out, kOutMaster | kOutSlices, 1.0, spec);
        prod_terms(op.out[0], M, T, 1.0);
        op.out[0].c = tanh_coef(k);
        scl[out] = op.out[0].s;
    };
    if (sub == kFtStart) {
        // Y = x^2: Y~ = v + (d_x[i] + d_x[j]) x~,  d_Y = d_x^2 + v_ii
        begin_op(op, Z, Z, Z, -1, 1.0 / (static_cast<double>(scl[Z]) * scl[Z]));
        op.nout = 3;
        out_d(op.out[0], M, kOutMaster | kOutSlices, 1.0, r2);
        set_e(op.out[0], Z, 0.0, 1.0, 1.0, -1, 0.0, 0.0, 0.0);
        set_d(op.out[0], 0.0, Z, Z, 1.0, 0.0, 0.0);
        // T5 = c4 I + c5 Y
        const double c4 = tanh_coef(4), c5 = tanh_coef(5);
        out_d(op.out[1], N, kOutMaster | kOutSlices, c5, tb[5]);
        set_e(op.out[1], Z, 0.0, c5, c5, -1, 0.0, 0.0, 0.0);
        set_d(op.out[1], c4, Z, Z, c5, 0.0, 0.0);
        // copy of x
        out_d(op.out[2], X, kOutMaster | kOutSlices, 0.0, r);
        set_e(op.out[2], -1, 1.0, 0.0, 0.0, -1, 0.0, 0.0, 0.0);
        set_d(op.out[2], 0.0, Z, -1, 0.0, 1.0, 0.0);
        scl[M] = op.out[0].s;
        scl[N] = op.out[1].s;
        scl[X] = op.out[2].s;
        st->ft_sub = kFtPoly1;
        st->ft_last_mat = M;
    } else if (sub == kFtPoly1) {
        horner(N, W0, 3, tb[4]);
        st->ft_sub = kFtPoly2;
        st->ft_last_mat = W0;
    } else if (sub == kFtPoly2) {
        horner(W0, N, 2, tb[3]);
        st->ft_sub = kFtPoly3;
        st->ft_last_mat = N;
    } else if (sub == kFtPoly3) {
        horner(N, W0, 1, tb[2]);
        st->ft_sub = kFtPoly4;
        st->ft_last_mat = W0;
    } else if (sub == kFtPoly4) {
        horner(W0, N, 0, tb[1]);
        st->ft_sub = kFtPoly5;
        st->ft_last_mat = N;
    } else {
        // z0 = x P: E1 = P~ (row d_x), E2 = x~ (column d_P); |tanh x| <= |x|
        begin_op(op, X, N, N, X, 1.0 / (static_cast<double>(scl[X]) * scl[N]));
        op.nout = 1;
        out_d(op.out[0], Z, kOutMaster | kOutSlices, 1.0, r);
        prod_terms(op.out[0], X, N, 1.0);
        scl[Z] = op.out[0].s;
        op.part_out = 0;  // tr z0 and ||z0||_F^2 for the first decision
        st->ft_sub = kFtPoly6;
        st->ft_last_mat = Z;
    }
}

// Newton-Schulz steps W <- W (2 I - M W) after the closed-form first
// iterate run until the residual bound, r0^2 after that iterate (r0 =
// (m_max - m_min)/(m_max + m_min)) and squared by every step, falls below
// 3e-8.  The residual leaves each eigenvalue's z'' short by at most that
// fraction.  The doubling map never raises a relative error
// (d ln f / d ln z = (1 - z^2)/(1 + z^2) <= 1) and nearly erases it where |z|
// is close to 1, so the saturated states carry only the last stage's
// residual, D moves by about half of it, and tr D is restored by the closing
// shift steps: 3e-8 stays well inside the 1e-6 (D) and 1e-7 (band energy per
// electron) tolerances.
//
// The iteration corrects itself: a step's rounding error e only leaves a
// residual of about e for the next step to square.  So under the mixed
// policy the pairs whose input bound is still >= 0.05 run as single-FP16
// products (one MMA instead of three), which leave a residual of at most
// about 2^-10 kappa(M) <= 4e-3 (kappa <= 2 here) besides the square of their
// input; the remaining pairs are split-FP16 and bring the bound under 3e-8.
constexpr double kNsTarget = 3e-8, kNsSingleAbove = 0.05, kNsSingleFloor = 4e-3;
// largest Newton logit shift folded into a doubling without a shift-only step
constexpr double kFoldMax = 0.4;
constexpr int kNsMaxSteps = 12;

__device__ double ns_residual0(double mmin, double mmax) {
    const double r0 = (mmax - mmin) / (mmax + mmin);
    return r0 * r0;
}

__device__ void control_fermi(SolveState *st, double tr0, double sq0, double tr1) {
    const int n = st->n;
    const double nn = static_cast<double>(n);
    const double ne = st->ne;
    ProdOp &op = st->op;
    const int sub = st->ft_sub;
    double *sc = st->sc, *fb = st->fb;
    float *scl = st->scl;
    const int Z = kMatZ, N = kMatN, M = kMatM, R = kMatR, WS = kMatW0;  // WS: W's scalar slot

    if (st->iter < kHistRows) {
        // stage, last step, tr D - N_e (when z is fresh), mu estimate, W's
        // identity part, ||output~||_F of the last step
        double *h = st->hist[st->iter];
        h[0] = st->ft_stage;
        h[1] = sub;
        h[2] = 0.5 * (nn - (nn * sc[Z] + tr0)) - ne;
        h[3] = st->mu_t;
        h[4] = sc[WS];
        h[5] = sqrt(fmax(sq0, 0.0));
    }
    if (sub == kFtFinal) {
        // the final product wrote D0 and Q: keep their exact traces
        st->tr_d0 = tr0;
        st->tr_q = tr1;
        st->done = 1;
        st->kind = kNone;
        return;
    }
    if (st->iter >= st->max_iters) {
        st->status = -3;
        st->done = 1;
        st->kind = kNone;
        return;
    }
    // The partials carry the exact ||A~||_F of the step's reported output:
    // replace the a-priori bound (triangle inequalities would compound over
    // the Newton-Schulz steps and push the slice scales out of range).
    if (sub != kFtStart) fb[st->ft_last_mat] = sqrt(fmax(sq0, 0.0));
    st->iter += 1;
    const int W = st->wcur;

    // ---- z0 = tanh(x) by the polynomial start
    if (sub == kFtStart || (sub >= kFtPoly1 && sub <= kFtPoly5)) {
        control_fermi_start(st, sub);
        return;
    }

    // ---- Newton-Schulz inner steps
    if (sub == kFtSquare || sub == kFtShiftElem || sub == kFtWR) {
        if (sub == kFtWR) {
            st->ft_j += 1;
            const double r2 = st->ns_r * st->ns_r;
            st->ns_r = st->ns_single ? fmax(r2, kNsSingleFloor) : r2;
        }
        if (st->ns_r > kNsTarget && st->ft_j < kNsMaxSteps) {
            // R = M W; spec(M W) in [1 - r, 1 + r]
            st->ns_single = (st->prec == kPrecMixed && st->ns_r >= kNsSingleAbove) ? 1 : 0;
            st->kind = st->ns_single ? kTcSingle : kTcSplit;
            begin_op(op, M, W, W, M, 1.0 / (static_cast<double>(scl[M]) * scl[W]));
            op.nout = 1;
            out_d(op.out[0], R, kOutMaster | kOutSlices, 1.0, 1.0 + st->ns_r);
            prod_terms(op.out[0], M, W, 1.0);
            scl[R] = op.out[0].s;
            st->ft_sub = kFtMW;
            st->ft_last_mat = R;
        } else {
            // z'' = N W = tanh(...) up to the residual: spec in [-1 - r, 1 + r]
            st->kind = kTcSplit;
            begin_op(op, N, W, W, N, 1.0 / (static_cast<double>(scl[N]) * scl[W]));
            op.nout = 1;
            out_d(op.out[0], Z, kOutMaster | kOutSlices, 1.0, 1.0 + st->ns_r);
            prod_terms(op.out[0], N, W, 1.0);
            scl[Z] = op.out[0].s;
            op.part_out = 0;  // tr z and ||z||_F^2 for the next Newton step on mu
            st->ft_sub = kFtNW;
            st->ft_last_mat = Z;
        }
        return;
    }
    if (sub == kFtMW) {
        // W' = 2 W - W R:  W'~ = (2 - d_R[j]) W~ - d_W[i] R~ - v,
        // d_W' = 2 d_W - d_W d_R - v_ii;  W' = (1 - r'(m)) / m with |r'| <= r
        // on the spectrum [mmin, mmax] of M
        const int Wn = (W == kMatW0) ? kMatW1 : kMatW0;
        st->kind = st->ns_single ? kTcSingle : kTcSplit;
        begin_op(op, W, R, W, R, 1.0 / (static_cast<double>(scl[W]) * scl[R]));
        op.nout = 1;
        out_d(op.out[0], Wn, kOutMaster | kOutSlices, -1.0, (1.0 + st->ns_r) / st->ns_mmin);
        set_e(op.out[0], R, 2.0, 0.0, -1.0, W, 0.0, -1.0, 0.0);
        set_d(op.out[0], 0.0, W, R, -1.0, 2.0, 0.0);
        scl[Wn] = op.out[0].s;
        st->wcur = Wn;
        st->ft_sub = kFtWR;
        st->ft_last_mat = Wn;
        return;
    }

    // ---- z is fresh (after X0 or after N W): decide the next step
    // Phases of the chemical-potential control:
    //   A  plain doublings while z is nearly linear in H (rms of z < 0.25):
    //      tr D stays near n/2 whatever mu is, so nothing is tracked yet;
    //   B  (entered when z turns nonlinear) shift-only Newton steps until
    //      tr D = N_e at the current temperature;
    //   C  doublings with the Newton shift of the current trace error folded
    //      in (mu(T) moves by less than kT per halving of T from here on);
    //      a large error falls back to shift-only steps;
    //   D  after the last doubling, shift-only Newton steps until
    //      |tr D - N_e| <= 1e-3, then the final trace-exact product.
    // diagonal form: the partials are tr z and ||z||_F^2 themselves
    const double trz = tr0;
    const double zz = sq0;
    fb[Z] = sqrt(fmax(sq0, 0.0));
    const double trD = 0.5 * (nn - trz);
    const double slope = 0.5 * (nn - zz);  // d tr D / d b with b the logit shift
    double b = (slope > 1e-300) ? (ne - trD) / slope : 0.0;
    const double dN = ne - trD;
    const bool stages_done = st->ft_stage >= st->ft_m;
    const double z_rms = sqrt(fmax(zz, 0.0) / nn);
    if (st->ft_phase == 0 && (z_rms >= 0.25 || stages_done)) st->ft_phase = 1;
    bool shift_only;
    if (stages_done) {
        shift_only = true;
    } else if (st->ft_phase == 0) {
        shift_only = false;
        b = 0.0;
    } else {
        // large errors (entering phase B, or after a big drift) are removed by
        // shift-only steps; small ones ride along with the next doubling.
        // "Small" is in the logit: a Newton step |b| <= kFoldMax is accurate
        // to a few per cent (the trace is smooth in b on that scale), and the
        // next stage measures and corrects what it missed, so nothing is
        // gained by verifying it first with a shift-only step.
        shift_only = fabs(b) > kFoldMax && st->ft_shifts < 6;
    }
    if (stages_done && (fabs(dN) <= 1e-3 || st->ft_shifts >= 6)) {
        // ---- final product: D0 = (I - z)/2 and Q = (I - z^2)/4 in FP64
        //   D0: -z~/2 off the diagonal, (1 - d_z)/2 on it
        //   Q:  -(v + (d_z[i] + d_z[j]) z~)/4 off it, (1 - d_z^2 - v_ii)/4 on it
        st->kind = kTcSplit;
        begin_op(op, Z, Z, Z, -1, 1.0 / (static_cast<double>(scl[Z]) * scl[Z]));
        op.nout = 2;
        out_d(op.out[0], Z, kOutF64a, 0.0, 1.0);
        set_e(op.out[0], -1, -0.5, 0.0, 0.0, -1, 0.0, 0.0, 0.0);
        set_d(op.out[0], 0.5, Z, -1, 0.0, -0.5, 0.0);
        out_d(op.out[1], Z, kOutF64b, -0.25, 1.0);
        set_e(op.out[1], Z, 0.0, -0.25, -0.25, -1, 0.0, 0.0, 0.0);
        set_d(op.out[1], 0.25, Z, Z, -0.25, 0.0, 0.0);
        op.part_out = 0;
        st->ft_sub = kFtFinal;
        return;
    }
    const double beta_k = st->beta0 * ldexp(1.0, st->ft_stage);  // z = tanh(beta_k (H - mu)/2)
    // spectral radius of z: |tanh(beta_k (lambda - mu)/2)| over the bound
    // interval (the margin covers the expansion's rounding).  Early stages
    // have small z, so M is close to I and Newton-Schulz needs few or no steps.
    const double rad = fmax(fabs(st->emax - st->mu_t), fabs(st->emin - st->mu_t));
    const double rho = fmin(1.0, tanh(0.5 * beta_k * rad) * (1.0 + 1e-6) + 1e-6);
    if (!shift_only && st->ft_phase != 0) {
        // The doubling halves T, and mu(T) moves with it.  mu(beta_k) is the
        // current estimate corrected by the Newton step; from the second
        // tracked stage on, the next stage's mu is predicted from the last
        // two: mu(T) - mu(0) goes as T^2 at low T (Sommerfeld), so each
        // halving of T quarters the change, mu_{k+1} - mu_k = (mu_k - mu_{k-1})/4.
        // Folding that drift into the shift spares the shift-only steps that
        // would otherwise correct it at the next stage.
        const double bn = fmax(-0.5, fmin(0.5, b));
        const double mu_k = st->mu_t + 2.0 * bn / beta_k;
        if (st->mu_nconv >= 1) b = bn + 0.5 * beta_k * 0.25 * (mu_k - st->mu_prev);
        st->mu_prev = mu_k;
        st->mu_nconv += 1;
    }
    b = shift_only ? fmax(-1.0, fmin(1.0, b)) : fmax(-0.5, fmin(0.5, b));
    const double t = tanh(b);
    st->ft_t = t;
    st->mu_t += 2.0 * b / beta_k;
    st->ft_j = 0;
    st->ns_single = 0;
    if (!shift_only) {
        st->ft_shifts = 0;
        // ---- shift + double, with z = diag(d) + z~ and v = z~ z~:
        //   z^2 = diag(d^2 + v_ii) + (d[i] + d[j]) z~ + v
        //   M = (1 + t^2)(I + z^2) - 4 t z,  N = 2 ((1 + t^2) z - t (I + z^2)),
        //   W1 = 2 w0 I - w0^2 M (first Newton-Schulz iterate)
        const double t2 = t * t, tp = 1.0 + t2;
        // spectrum of M: m(x) = (1 + t^2)(1 + x^2) - 4 t x = (1 - t x)^2 + (x - t)^2
        // over x in [-rho, rho]; a convex quadratic with its minimum at 2t/(1 + t^2)
        const double m_p = tp * (1.0 + rho * rho) - 4.0 * t * rho;
        const double m_m = tp * (1.0 + rho * rho) + 4.0 * t * rho;
        const double mmax = fmax(m_p, m_m);
        const double mmin = (fabs(2.0 * t / tp) <= rho) ? (1.0 - t2) * (1.0 - t2) / tp : fmin(m_p, m_m);
        const double w0 = 2.0 / (mmin + mmax);
        st->w0 = w0;
        st->ns_r = ns_residual0(mmin, mmax);
        st->ns_mmin = mmin;
        st->ns_mmax = mmax;
        const double sN = 2.0 * (tp * rho + fabs(t) * (1.0 + rho * rho));  // ||N||_2
        const double sW = fmax(fabs(2.0 * w0 - w0 * w0 * mmax), fabs(2.0 * w0 - w0 * w0 * mmin));
        const double w2 = w0 * w0;
        st->kind = kTcSplit;
        begin_op(op, Z, Z, Z, -1, 1.0 / (static_cast<double>(scl[Z]) * scl[Z]));
        op.nout = 3;
        out_d(op.out[0], M, kOutMaster | kOutSlices, tp, mmax);
        set_e(op.out[0], Z, -4.0 * t, tp, tp, -1, 0.0, 0.0, 0.0);
        set_d(op.out[0], tp, Z, Z, tp, -4.0 * t, 0.0);
        out_d(op.out[1], N, kOutMaster | kOutSlices, -2.0 * t, sN);
        set_e(op.out[1], Z, 2.0 * tp, -2.0 * t, -2.0 * t, -1, 0.0, 0.0, 0.0);
        set_d(op.out[1], -2.0 * t, Z, Z, -2.0 * t, 2.0 * tp, 0.0);
        out_d(op.out[2], W, kOutMaster | kOutSlices, -w2 * tp, sW);
        set_e(op.out[2], Z, 4.0 * t * w2, -w2 * tp, -w2 * tp, -1, 0.0, 0.0, 0.0);
        set_d(op.out[2], 2.0 * w0 - w2 * tp, Z, Z, -w2 * tp, 4.0 * t * w2, 0.0);
        scl[M] = op.out[0].s;
        scl[N] = op.out[1].s;
        scl[W] = op.out[2].s;
        st->ft_stage += 1;
        st->ft_sub = kFtSquare;
        st->ft_last_mat = M;
    } else {
        // ---- shift only: N = z - t I, M = I - t z, spectrum of M in [1 - |t| rho, 1 + |t| rho];
        // no product: M~ = -t z~, d_M = 1 - t d;  N~ = z~, d_N = d - t;
        // W1~ = w0^2 t z~, d_W1 = 2 w0 - w0^2 + w0^2 t d
        const double mmin = 1.0 - fabs(t) * rho, mmax = 1.0 + fabs(t) * rho;
        const double w0 = 2.0 / (mmin + mmax);
        st->w0 = w0;
        st->ns_r = ns_residual0(mmin, mmax);
        st->ns_mmin = mmin;
        st->ns_mmax = mmax;
        const double w2 = w0 * w0;
        st->kind = kTcElem;
        begin_op(op, Z, Z, Z, -1, 0.0);
        op.nout = 3;
        out_d(op.out[0], M, kOutMaster | kOutSlices, 0.0, mmax);
        set_e(op.out[0], -1, -t, 0.0, 0.0, -1, 0.0, 0.0, 0.0);
        set_d(op.out[0], 1.0, Z, -1, 0.0, -t, 0.0);
        out_d(op.out[1], N, kOutMaster | kOutSlices, 0.0, rho + fabs(t));
        set_e(op.out[1], -1, 1.0, 0.0, 0.0, -1, 0.0, 0.0, 0.0);
        set_d(op.out[1], -t, Z, -1, 0.0, 1.0, 0.0);
        out_d(op.out[2], W, kOutMaster | kOutSlices, 0.0, fmax(fabs(2.0 * w0 - w2 * mmax), fabs(2.0 * w0 - w2 * mmin)));
        set_e(op.out[2], -1, w2 * t, 0.0, 0.0, -1, 0.0, 0.0, 0.0);
        set_d(op.out[2], 2.0 * w0 - w2, Z, -1, 0.0, w2 * t, 0.0);
        scl[M] = op.out[0].s;
        scl[N] = op.out[1].s;
        scl[W] = op.out[2].s;
        st->ft_shifts += 1;
        st->ft_sub = kFtShiftElem;
        st->ft_last_mat = M;
    }
}

}  // namespace

namespace {

__device__ void control_one(const MmaProb &pr, const DevCtl *ctl) {
    SolveState *st = pr.st;
    if (st->done) return;
    if (ctl && *reinterpret_cast<const volatile int *>(&ctl->err) != 0) {
        // a kernel of this run gave up a bounded wait: its outputs are not
        // trustworthy, so the expansion stops here
        if (threadIdx.x == 0) {
            st->status = -4;  // FE_ETIMEOUT
            st->done = 1;
            st->kind = kNone;
        }
        return;
    }

    // number of partial slots written by the previous producer
    int nparts;
    if (st->kind == kNone) nparts = kInitBlocks;
    else if (st->kind == kFp64 || st->kind == kDf) nparts = pr.ntiles64;
    else if (st->kind == kDigit) nparts = pr.ntilesD;
    else nparts = pr.ntiles;

    __shared__ double s_a[256], s_b[256], s_c[256], s_d[256];
    const int t = threadIdx.x;
    double a = 0, b = 0, c = 0, d = 0;
    for (int k = t; k < nparts; k += blockDim.x) {
        const double *slot = pr.part + static_cast<size_t>(k) * kPartStride;
        a += slot[0];
        b += slot[1];
        c += slot[2];
        d += slot[3];
    }
    s_a[t] = a; s_b[t] = b; s_c[t] = c; s_d[t] = d;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            s_a[t] += s_a[t + o];
            s_b[t] += s_b[t + o];
            s_c[t] += s_c[t + o];
            s_d[t] += s_d[t + o];
        }
        __syncthreads();
    }
    if (t != 0) return;
    if (st->bad_input) {
        st->status = -1;  // FE_EINVAL
        st->done = 1;
        st->kind = kNone;
        return;
    }
    if (st->chk_left > 0 || st->chk) {
        control_check(st, s_a[0], s_b[0]);
        return;
    }
    if (st->method == kMethodFermi) control_fermi(st, s_a[0], s_b[0], s_c[0]);
    else if (st->method == kMethodTrfoe) control_trfoe(st, s_a[0], s_b[0]);
    else control_sp2(st, s_a[0], s_b[0], s_d[0]);
    // the kind of every step issued (step k runs in the k-th pass of the step loop)
    if (st->nctl < kKindLog) st->kind_log[st->nctl] = static_cast<unsigned char>(st->done ? kNone : st->kind);
    st->nctl += 1;
}

}  // namespace

__global__ void k_control(const MmaProb *probs, int nprobs, const DevCtl *ctl, StepFlags *flags,
                          cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_tc,
                          cudaGraphConditionalHandle h_fp64, cudaGraphConditionalHandle h_digit,
                          unsigned hvalid) {
    const int p = blockIdx.x;
    if (p < nprobs) control_one(probs[p], ctl);
    if (!flags || threadIdx.x != 0) return;
    // Inside the step graph: collect what the next step needs over all
    // problems; the block that finishes last sets the graph's conditions
    // (loop on while any problem is active; one switch per kernel family).
    unsigned bits = 0;
    if (p < nprobs) {
        const SolveState *st = probs[p].st;
        const int kind = *reinterpret_cast<const volatile int *>(&st->kind);
        if (!*reinterpret_cast<const volatile int *>(&st->done)) {
            bits |= kStepActive;
            if (kind == kTcSingle || kind == kTcSplit || kind == kTcElem || kind == kTcDelta) bits |= kStepTc;
            if (kind == kFp64 || kind == kDf) bits |= kStepFp64;
            if (kind == kDigit) bits |= kStepDigit;
        }
    }
    if (bits) atomicOr(&flags->mask, bits);
    __threadfence();
    if (atomicAdd(&flags->count, 1u) != static_cast<unsigned>(gridDim.x) - 1u) return;
    __threadfence();
    const unsigned m = atomicExch(&flags->mask, 0u);
    atomicExch(&flags->count, 0u);
    const bool on = (m & kStepActive) != 0;
    // hvalid: which handles exist in this graph (bit = the family's StepBits)
    if (hvalid & kStepActive) cudaGraphSetConditional(h_loop, on ? 1u : 0u);
    if (hvalid & kStepTc) cudaGraphSetConditional(h_tc, (on && (m & kStepTc)) ? 1u : 0u);
    if (hvalid & kStepFp64) cudaGraphSetConditional(h_fp64, (on && (m & kStepFp64)) ? 1u : 0u);
    if (hvalid & kStepDigit) cudaGraphSetConditional(h_digit, (on && (m & kStepDigit)) ? 1u : 0u);
    flags->n_body += 1;
    if (on) {
        flags->n_tc += (m & kStepTc) ? 1u : 0u;
        flags->n_fp64 += (m & kStepFp64) ? 1u : 0u;
        flags->n_digit += (m & kStepDigit) ? 1u : 0u;
    }
}

}  // namespace fe
