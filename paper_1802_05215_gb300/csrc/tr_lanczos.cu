// Filtered thick-restart Lanczos with locking (Algorithm 2) as a per-slice state machine.
//
// A SliceSolver owns the locked set U and the basis Q of one slice and the small projected
// matrix T on the host.  Its step is split in two: input() names the vector that must be
// filtered next (q_i, or q_{l+1} for the special TR step) and consume(y) takes y = rho(A) q and
// finishes the step (three-term recurrence, full reorthogonalisation, early-restart test, and,
// when the cycle ends, the restart with Ritz vectors, locking and the next TR set).  A single
// slice is driven with the one-vector filter kernel; several slices of one matrix are driven
// in lockstep, with all their filter applications of a step done by the multi-slice block
// kernel (one pass over the matrix per degree for all slices).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "evsl_internal.h"

namespace {

constexpr double DGKS_ETA2 = 0.5;  // (1/sqrt(2))^2: second Gram-Schmidt pass when ||z'||^2 < 0.5 ||z||^2
constexpr int POLISH_BLOCKS = 3;            // Krylov blocks per polish cycle after an FP32 run
constexpr int POLISH_CYCLES = 6;            // polish cycles at most
constexpr double POLISH_SELECT = 0.9;       // Ritz values of rho kept for the A projection: mu >= 0.9 bar
constexpr double POLISH_RHO_RES = 1e-3;     // ... whose vectors have ||rho y - mu y|| <= 1e-3 |mu|
constexpr double MIXED_TOL_LOCK_MAX = 1e-4; // loosest locking level of the FP32 phase

enum Scal { ALPHA = 0, NRM_BEFORE = 1, NRM_AFTER = 2, NRM_Y = 3, TMP = 4, H = 16 };

int d2h(evsl_ctx *c, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "device-to-host copy");
}

int h2d(evsl_ctx *c, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "host-to-device copy");
}

int d2d(evsl_ctx *c, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? EVSL_OK : ctx_cuda(c, e, "device-to-device copy");
}

float ev_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

class SliceSolver {
public:
    // nonrestart: the non-restart variant (ChebLanNr): one basis of at most m vectors, no locking
    // or thick restart; see end_cycle_nr
    SliceSolver(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts &o,
                int m, int cap, bool right_closed, bool nonrestart = false)
        : c_(c), n_(c->A.n), a_(a), b_(b), pol_(pol), o_(o), cap_(cap), right_closed_(right_closed),
          nonrestart_(nonrestart)
    {
        m_ = std::min<int64_t>(m, n_);
        maxit_ = nonrestart ? m_ : (o.maxit > 0 ? o.maxit : 20 * m_);
        ncycle_ = o.ncycle > 0 ? o.ncycle : 10;
        tol_ = o.tol > 0 ? o.tol : 1e-8;
        tau1_ = o.tau1 > 0 ? o.tau1 : 1e-10;
        bar_ = pol->bar;
        normA_ = std::max(std::fabs(pol->lmin), std::fabs(pol->lmax));
        // FP32 filter: phase 1 locks at the FP32-reachable level in a slice widened by the
        // corresponding eigenvalue error; the FP64 polish at the end decides membership and tol
        mixed_ = (o.prec == EVSL_FP32);
        tol_lock_ = mixed_ ? std::max(tol_, 1e-6) : tol_;
        widen_ = mixed_ ? tol_lock_ * normA_ : 0.0;
        const char *venv = getenv("EVSL_VERBOSE");
        verbose_ = venv && venv[0] == '1';
    }

    ~SliceSolver()
    {
        ctx_free(c_, U_, sizeof(double) * n_ * cap_);
        ctx_free(c_, Q_, sizeof(double) * n_ * (m_ + 1));
        ctx_free(c_, sc_, sizeof(double) * nsc_);
        for (cudaEvent_t e : {e0_, e1_, e2_})
            if (e) cudaEventDestroy(e);
    }

    int init()
    {
        nsc_ = H + (size_t)cap_ + m_ + 1 + 8;
        EVSL_TRY(ctx_alloc(c_, (void **)&U_, sizeof(double) * n_ * cap_));
        EVSL_TRY(ctx_alloc(c_, (void **)&Q_, sizeof(double) * n_ * (m_ + 1)));
        EVSL_TRY(ctx_alloc(c_, (void **)&sc_, sizeof(double) * nsc_));
        h_ = sc_ + H;
        cudaEventCreate(&e0_);
        cudaEventCreate(&e1_);
        cudaEventCreate(&e2_);
        T_.assign((size_t)(m_ + 1) * (m_ + 1), 0.0);
        EVSL_TRY(fresh_vector(fresh_index_++, Q_, 0, 0));
        l_ = 0;
        begin_cycle();
        return EVSL_OK;
    }

    bool done() const { return done_; }

    // Polynomial filtered subspace iteration (ChebSI) with a block of nv = m vectors held in the
    // basis array, at most `maxpass` Rayleigh-Ritz passes.  V starts as nv seeded random vectors,
    // orthonormalised; each pass forms W = rho(Ahat) V, and when V holds the previous pass's Ritz
    // vectors, mu_j = v_j^T w_j is the filter's Rayleigh quotient of v_j: a vector made only of
    // eigenvectors outside the slice has mu < bar, an in-slice eigenvector mu >= bar.  The run
    // stops when every in-slice Ritz pair with mu >= bar meets tol; otherwise W is orthonormalised
    // (dropped dependent directions are replaced by fresh seeded vectors) and Rayleigh-Ritz with A
    // gives the next V.  The converged in-slice pairs become the result (EVSL_ERR_NOCONV after
    // maxpass passes with wanted pairs unconverged, EVSL_ERR_CAPACITY beyond cap).
    int run_si(int maxpass)
    {
        const int nv = m_;
        const int nc = std::min(nv, 64);
        int st = EVSL_OK;
        double *V = Q_;
        double *W = (double *)ctx_ws(c_, WS_POL_W, sizeof(double) * n_ * nv, &st);
        if (st) return st;
        double *B = (double *)ctx_ws(c_, WS_POL_B, sizeof(double) * n_ * 2 * nc, &st);
        if (st) return st;
        double *mud = (double *)ctx_ws(c_, WS_POL_H, sizeof(double) * ((size_t)nv + 8), &st);
        if (st) return st;
        for (int j = 0; j < nv; j++)
            EVSL_TRY(fill_uniform_f64(c_, n_, o_.seed, SM_STREAM_LANCZOS, fresh_index_++, V + (int64_t)j * n_));
        int kv = 0;
        EVSL_TRY(orthonormalize(V, nv, W, &kv));
        EVSL_TRY(refill_block(V, kv, nv, W, &kv));
        std::vector<double> th, r2, mu;
        bool ritz = false;
        for (int pass = 1; pass <= maxpass + 1; pass++) {
            cudaEventRecord(e0_, c_->stream);
            for (int j0 = 0; j0 < kv; j0 += nc) {
                const int mcols = std::min(nc, kv - j0);
                const int64_t o = (int64_t)j0 * n_;
                EVSL_TRY(filter_apply_dev(c_, pol_, mcols, V + o, W + o, EVSL_FP64, B, B + (int64_t)mcols * n_, nullptr));
            }
            cudaEventRecord(e1_, c_->stream);
            cudaEventSynchronize(e1_);
            t_filter_ += ev_ms(e0_, e1_) * 1e-3;
            nmv_ += (int64_t)pol_->deg * kv;
            if (ritz) {
                EVSL_TRY(coldot(c_, n_, kv, V, n_, W, n_, mud));
                mu.assign(kv, 0.0);
                EVSL_TRY(d2h(c_, mu.data(), mud, sizeof(double) * kv));
                bool all = true;
                for (int j = 0; j < kv; j++)
                    if (in_slice(th[j]) && mu[j] >= bar_ && std::sqrt(std::max(0.0, r2[j])) / normA_ > tol_)
                        all = false;
                if (verbose_) {
                    int nin = 0, nconv = 0;
                    for (int j = 0; j < kv; j++)
                        if (in_slice(th[j])) {
                            nin++;
                            nconv += std::sqrt(std::max(0.0, r2[j])) / normA_ <= tol_;
                        }
                    fprintf(stderr, "[evsl] si pass %d: block=%d in_slice=%d converged=%d%s\n", pass - 1, kv, nin,
                            nconv, all ? " (done)" : "");
                }
                if (all || pass == maxpass + 1) {
                    std::vector<int> keep;
                    for (int j = 0; j < kv; j++) {
                        const double rj = std::sqrt(std::max(0.0, r2[j])) / normA_;
                        if (!in_slice(th[j]) || rj > tol_) continue;
                        if ((int)keep.size() >= cap_) {
                            status_ = EVSL_ERR_CAPACITY;
                            break;
                        }
                        keep.push_back(j);
                        lam_l_.push_back(th[j]);
                        res_l_.push_back(rj);
                    }
                    if (!all && status_ == EVSL_OK) status_ = EVSL_ERR_NOCONV;
                    if (!keep.empty()) {
                        int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * (keep.size() + 8), &st);
                        if (st) return st;
                        EVSL_TRY(h2d(c_, idx, keep.data(), sizeof(int) * keep.size()));
                        EVSL_TRY(gather_cols(c_, n_, (int)keep.size(), V, n_, idx, U_, n_));
                    }
                    nlock_ = (int)keep.size();
                    its_ = pass - 1;
                    break;
                }
            }
            cudaEventRecord(e0_, c_->stream);
            int kw = 0;
            EVSL_TRY(orthonormalize(W, kv, V, &kw));
            EVSL_TRY(refill_block(W, kw, kv, V, &kw));
            int sweeps = 0;
            EVSL_TRY(rayleigh_ritz(W, kw, V, th, r2, &sweeps));
            kv = kw;
            ritz = true;
            nrestart_++;
            cudaEventRecord(e1_, c_->stream);
            cudaEventSynchronize(e1_);
            t_restart_ += ev_ms(e0_, e1_) * 1e-3;
            its_ = pass;
        }
        done_ = true;
        return EVSL_OK;
    }
    int status() const { return status_; }
    const evsl_polfilt *pol() const { return pol_; }

    // the vector the next step filters
    const double *input() const { return Q_ + (int64_t)(tr_pending_ ? l_ : i_) * n_; }

    // one finished Lanczos step: y = rho(A) input() (y may be overwritten); t_filter_s is the
    // device time the filter took
    int consume(double *y, double t_filter_s)
    {
        t_filter_ += t_filter_s;
        nmv_ += pol_->deg;
        its_++;
        cudaEventRecord(e1_, c_->stream);
        if (tr_pending_) {
            EVSL_TRY(tr_step(y));
            tr_pending_ = false;
            k_ = l_ + 1;
            lstart_ = k_;
            i_ = k_;
            if (i_ >= m_) return end_cycle();
            return EVSL_OK;
        }
        bool stop_cycle = false;
        EVSL_TRY(lanczos_step(y, &stop_cycle));
        if (nonrestart_) {
            if (stop_cycle || i_ + 1 >= m_) EVSL_TRY(end_cycle_nr(i_ + 1 >= m_));
            if (!done_) i_++;
            return EVSL_OK;
        }
        if (stop_cycle || its_ > maxit_ || i_ + 1 >= m_) return end_cycle();
        i_++;
        return EVSL_OK;
    }

    int finish(int *nev, double *lam, double *res, double *Y, evsl_stats *st, double t_total)
    {
        if (mixed_ && nlock_ > 0) {
            cudaEventRecord(e0_, c_->stream);
            const int pst = polish();
            if (pst == EVSL_ERR_NOMEM) {
                // no room for the polish's block workspaces under the HBM budget: the FP64
                // re-solve below needs only a basis like the one this run already held
                c_->err.clear();
                status_ = EVSL_ERR_NOCONV;
            } else if (pst != EVSL_OK) {
                return pst;
            }
            cudaEventRecord(e1_, c_->stream);
            cudaEventSynchronize(e1_);
            t_restart_ += ev_ms(e0_, e1_) * 1e-3;
            // the polish could not bring every in-slice pair to tol: solve the slice again with
            // the FP64 filter, so that the result is the plain FP64 method's
            if (status_ == EVSL_ERR_NOCONV) EVSL_TRY(resolve_fp64());
        }
        std::vector<int> perm(nlock_);
        std::iota(perm.begin(), perm.end(), 0);
        std::sort(perm.begin(), perm.end(), [&](int x, int y) { return lam_l_[x] < lam_l_[y]; });
        for (int i = 0; i < nlock_; i++) {
            lam[i] = lam_l_[perm[i]];
            res[i] = res_l_[perm[i]];
        }
        if (Y && nlock_ > 0) {
            cudaPointerAttributes attr;
            bool ydev = (cudaPointerGetAttributes(&attr, Y) == cudaSuccess) &&
                        (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
            cudaGetLastError();
            if (ydev) {
                int s = EVSL_OK;
                int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * (size_t)(nlock_ + 8), &s);
                if (s) return s;
                EVSL_TRY(h2d(c_, idx, perm.data(), sizeof(int) * nlock_));
                EVSL_TRY(gather_cols(c_, n_, nlock_, U_, n_, idx, Y, n_));
            } else {
                for (int i = 0; i < nlock_; i++) {
                    cudaError_t e = cudaMemcpyAsync(Y + (int64_t)i * n_, U_ + (int64_t)perm[i] * n_,
                                                    sizeof(double) * n_, cudaMemcpyDeviceToHost, c_->stream);
                    if (e != cudaSuccess) return ctx_cuda(c_, e, "eigenvector readback");
                }
            }
        }
        cudaError_t e = cudaStreamSynchronize(c_->stream);
        if (e != cudaSuccess) return ctx_cuda(c_, e, "chebLanTr outputs");
        *nev = nlock_;
        if (st) {
            st->niter = its_;
            st->nmv = nmv_;
            st->nrestart = nrestart_;
            st->npass = npass_;
            st->t_filter = t_filter_;
            st->t_orth = t_orth_;
            st->t_restart = t_restart_;
            st->t_total = t_total;
        }
        return EVSL_OK;
    }

private:
    double &t(int i, int j) { return T_[(size_t)j * (m_ + 1) + i]; }

    void begin_cycle()
    {
        std::fill(T_.begin(), T_.end(), 0.0);
        have_old_ = false;
        t_old_ = 0.0;
        prev_nabove_ = 0;
        if (l_ > 0) {
            for (int j = 0; j < l_; j++) {
                t(j, j) = trtheta_[j];
                t(j, l_) = trs_[j];
                t(l_, j) = trs_[j];
            }
            tr_pending_ = true;
        } else {
            tr_pending_ = false;
            k_ = 0;
            lstart_ = 0;
            i_ = 0;
        }
    }

    int cgs_pass(double *z, int nq, double *nrm2_dev)
    {
        EVSL_TRY(gemv_t2(c_, n_, U_, nlock_, Q_, nq, z, h_));
        return gemv_n2(c_, n_, U_, nlock_, Q_, nq, h_, z, nrm2_dev);
    }

    // fresh seeded vector in dst, orthogonalised (two passes) against U and Q[:, :nq]
    int fresh_vector(uint64_t index, double *dst, int nlock, int nq)
    {
        EVSL_TRY(fill_uniform_f64(c_, n_, o_.seed, SM_STREAM_LANCZOS, index, dst));
        for (int p = 0; p < 2; p++)
            if (nlock + nq > 0) {
                EVSL_TRY(gemv_t2(c_, n_, U_, nlock, Q_, nq, dst, h_));
                EVSL_TRY(gemv_n2(c_, n_, U_, nlock, Q_, nq, h_, dst, sc_ + TMP));
            }
        EVSL_TRY(coldot(c_, n_, 1, dst, n_, dst, n_, sc_ + TMP));
        double nr2 = 0;
        EVSL_TRY(d2h(c_, &nr2, sc_ + TMP, sizeof(double)));
        return scale_vec(c_, n_, dst, 1.0 / std::sqrt(nr2), nullptr);
    }

    // CGS with the DGKS test (at most two passes) of z against [U, Q[:, :nq]]
    int reorth(double *z, int nq, double nrm_before2, double *nrm2_out)
    {
        ProfGroup g;
        prof_begin(c_, EVSL_K_REORTH, &g);
        EVSL_TRY(cgs_pass(z, nq, sc_ + NRM_AFTER));
        npass_++;
        int launches = 4;
        double a2 = 0;
        EVSL_TRY(d2h(c_, &a2, sc_ + NRM_AFTER, sizeof(double)));
        if (a2 < DGKS_ETA2 * nrm_before2) {
            EVSL_TRY(cgs_pass(z, nq, sc_ + NRM_AFTER));
            npass_++;
            launches += 4;
            EVSL_TRY(d2h(c_, &a2, sc_ + NRM_AFTER, sizeof(double)));
        }
        prof_end(c_, &g, launches);
        *nrm2_out = a2;
        return EVSL_OK;
    }

    // q_{col+1} = z / beta, or a fresh vector after a breakdown; returns beta
    int next_vector(double *z, int col, double nrm2, double nrm_y2, double *beta_out)
    {
        double beta = std::sqrt(nrm2);
        double *qn = Q_ + (int64_t)(col + 1) * n_;
        if (beta <= 1e-13 * std::sqrt(nrm_y2)) {
            EVSL_TRY(fresh_vector(fresh_index_++, qn, nlock_, col + 1));
            beta = 0.0;
        } else {
            EVSL_TRY(scale_vec(c_, n_, z, 1.0 / beta, qn));
        }
        *beta_out = beta;
        return EVSL_OK;
    }

    void account_step()
    {
        cudaEventRecord(e2_, c_->stream);
        cudaEventSynchronize(e2_);
        t_orth_ += ev_ms(e1_, e2_) * 1e-3;
    }

    // special TR step on q_{l+1} = Q[:, l]: z = y - sum_j s_j u_j - alpha q_{l+1}
    int tr_step(double *y)
    {
        double *ql = Q_ + (int64_t)l_ * n_;
        EVSL_TRY(coldot(c_, n_, 1, y, n_, y, n_, sc_ + NRM_Y));
        EVSL_TRY(h2d(c_, h_, trs_.data(), sizeof(double) * l_));
        EVSL_TRY(gemv_n2(c_, n_, Q_, l_, nullptr, 0, h_, y, sc_ + TMP));
        EVSL_TRY(lan_three_term(c_, n_, y, nullptr, 0.0, ql, y, sc_ + ALPHA));
        EVSL_TRY(lan_sub_alpha(c_, n_, y, ql, sc_ + ALPHA, sc_ + NRM_BEFORE));
        double hs[4];
        EVSL_TRY(d2h(c_, hs, sc_, sizeof(double) * 4));
        double nrm2, beta;
        EVSL_TRY(reorth(y, l_ + 1, hs[1], &nrm2));
        EVSL_TRY(next_vector(y, l_, nrm2, hs[3], &beta));
        account_step();
        t(l_, l_) = hs[0];
        t(l_, l_ + 1) = beta;
        t(l_ + 1, l_) = beta;
        return EVSL_OK;
    }

    // ordinary step on column i: z = y - beta_i q_{i-1}; alpha = q_i^T z; z -= alpha q_i
    int lanczos_step(double *y, bool *stop_cycle)
    {
        const int i = i_;
        double *qi = Q_ + (int64_t)i * n_;
        EVSL_TRY(coldot(c_, n_, 1, y, n_, y, n_, sc_ + NRM_Y));
        const double bi = (i > 0) ? t(i - 1, i) : 0.0;
        EVSL_TRY(lan_three_term(c_, n_, y, i > 0 ? Q_ + (int64_t)(i - 1) * n_ : nullptr, bi, qi, y, sc_ + ALPHA));
        EVSL_TRY(lan_sub_alpha(c_, n_, y, qi, sc_ + ALPHA, sc_ + NRM_BEFORE));
        double hs[4];
        EVSL_TRY(d2h(c_, hs, sc_, sizeof(double) * 4));
        double nrm2, beta;
        EVSL_TRY(reorth(y, i + 1, hs[1], &nrm2));
        EVSL_TRY(next_vector(y, i, nrm2, hs[3], &beta));
        account_step();
        t(i, i) = hs[0];
        t(i, i + 1) = beta;
        t(i + 1, i) = beta;
        k_ = i + 1;
        if ((k_ - lstart_) % ncycle_ == 0) EVSL_TRY(early_restart_test(stop_cycle));
        return EVSL_OK;
    }

    // Every Ncycle steps: t = sum of the Ritz values >= bar (Sturm bisection on the arrowhead +
    // tridiagonal T).  Restart when t stalls (with a value above bar), or when nothing reached
    // bar at two consecutive tests after max(2 Ncycle, m/4) steps of the cycle.
    int early_restart_test(bool *stop)
    {
        const int k = k_, l = l_;
        std::vector<double> dd(k), ee(k, 0.0);
        for (int j = 0; j < k; j++) dd[j] = t(j, j);
        for (int j = 0; j < k; j++) {
            if (j < l) ee[j] = t(j, l);
            else if (j + 1 < k) ee[j] = t(j, j + 1);
        }
        int nbelow = host_count_below(k, l, dd.data(), ee.data(), bar_);
        int nabove = k - nbelow;
        double t_new = 0.0;
        if (nabove > 0) {
            double lo = 1e300, hi = -1e300, hub = 0.0;
            for (int j = 0; j < l; j++) hub += std::fabs(ee[j]);
            for (int j = 0; j < k; j++) {
                double rr;
                if (j < l) rr = std::fabs(ee[j]);
                else if (j == l) rr = hub + std::fabs(ee[j]);
                else rr = std::fabs(ee[j - 1]) + std::fabs(ee[j]);
                lo = std::min(lo, dd[j] - rr);
                hi = std::max(hi, dd[j] + rr);
            }
            std::vector<double> w(nabove);
            EVSL_TRY(bisect_eigs(c_, k, l, dd.data(), ee.data(), nbelow, k, lo, hi, w.data()));
            for (double v : w) t_new += v;
        }
        if (verbose_ && (k - lstart_) % (ncycle_ * 20) == 0)
            fprintf(stderr, "[evsl]   check its=%d k=%d nabove=%d t=%.12f\n", its_, k, nabove, t_new);
        if (have_old_ && nabove > 0 && std::fabs(t_new - t_old_) < tau1_ * std::max(1.0, std::fabs(t_new)))
            *stop = true;
        if (have_old_ && nabove == 0 && prev_nabove_ == 0 && k - lstart_ >= std::max(2 * ncycle_, m_ / 4))
            *stop = true;
        t_old_ = t_new;
        prev_nabove_ = nabove;
        have_old_ = true;
        return EVSL_OK;
    }

    // Ritz pairs of T_k with theta >= bar (largest first): their vectors Q S, normalised, go to
    // Yt (n x ncand0); lam = u^T A u, res = ||A u - lam u||^2, slast = last row of S.
    struct Cands {
        int ncand0 = 0, sweeps = 0;
        double betak = 0.0;
        std::vector<double> w, lam, res, slast;
        std::vector<int> order;
    };

    int ritz_candidates(int k, double *Yt, Cands *cd)
    {
        int st = EVSL_OK;
        const int zcols = std::min(m_, 128);
        double *Z = (double *)ctx_ws(c_, WS_LAN_Z, sizeof(double) * n_ * zcols, &st);
        if (st) return st;
        const int Mk = k + (k & 1) < 2 ? 2 : k + (k & 1);
        double *Vj = (double *)ctx_ws(c_, WS_LAN_T, sizeof(double) * (size_t)Mk * Mk, &st);
        if (st) return st;
        int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * (size_t)(2 * (m_ + 1) + 8), &st);
        if (st) return st;
        double *vd = (double *)ctx_ws(c_, WS_LAN_G, sizeof(double) * 3 * (size_t)(m_ + 1), &st);
        if (st) return st;
        double *lamd = vd, *resd = vd + (m_ + 1), *nrmd = vd + 2 * (m_ + 1);
        std::vector<double> Tk((size_t)k * k);
        cd->w.assign(k, 0.0);
        for (int j = 0; j < k; j++)
            for (int i = 0; i < k; i++) Tk[(size_t)j * k + i] = t(i, j);
        int ldv = 0;
        // jacobi_eig keeps its working copy in WS_LAN_S; the candidate block reuses it afterwards
        EVSL_TRY(jacobi_eig(c_, k, Tk.data(), cd->w.data(), Vj, &ldv, &cd->sweeps));
        double *Sd = (double *)ctx_ws(c_, WS_LAN_S, sizeof(double) * (size_t)Mk * Mk, &st);
        if (st) return st;
        cd->betak = t(k - 1, k);
        cd->order.resize(k);
        std::iota(cd->order.begin(), cd->order.end(), 0);
        const std::vector<double> &w = cd->w;
        std::sort(cd->order.begin(), cd->order.end(), [&](int x, int y) { return w[x] > w[y]; });
        int ncand0 = 0;
        while (ncand0 < k && w[cd->order[ncand0]] >= bar_) ncand0++;
        cd->ncand0 = ncand0;
        cd->lam.assign(ncand0, 0.0);
        cd->res.assign(ncand0, 0.0);
        cd->slast.assign(ncand0, 0.0);
        if (ncand0 == 0) return EVSL_OK;
        EVSL_TRY(h2d(c_, idx, cd->order.data(), sizeof(int) * ncand0));
        EVSL_TRY(gather_cols(c_, k, ncand0, Vj, ldv, idx, Sd, k));
        ProfGroup g;
        prof_begin(c_, EVSL_K_RITZ_GEMM, &g);
        EVSL_TRY(gemm_nn(c_, n_, ncand0, k, Q_, n_, Sd, k, Yt, n_));
        prof_end(c_, &g, 1);
        EVSL_TRY(coldot(c_, n_, ncand0, Yt, n_, Yt, n_, nrmd));
        EVSL_TRY(colscale_inv_sqrt(c_, n_, ncand0, Yt, nrmd));
        for (int j0 = 0; j0 < ncand0; j0 += zcols) {
            int nc = std::min(zcols, ncand0 - j0);
            EVSL_TRY(spmv_f64(c_, nc, Yt + (int64_t)j0 * n_, Z));
            EVSL_TRY(coldot(c_, n_, nc, Yt + (int64_t)j0 * n_, n_, Z, n_, lamd + j0));
            EVSL_TRY(colres2(c_, n_, nc, Z, Yt + (int64_t)j0 * n_, n_, lamd + j0, resd + j0));
        }
        EVSL_TRY(d2h(c_, cd->lam.data(), lamd, sizeof(double) * ncand0));
        EVSL_TRY(d2h(c_, cd->res.data(), resd, sizeof(double) * ncand0));
        cudaError_t e = cudaMemcpy2DAsync(cd->slast.data(), sizeof(double), Sd + (k - 1), sizeof(double) * k,
                                          sizeof(double), ncand0, cudaMemcpyDeviceToHost, c_->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c_->stream);
        if (e != cudaSuccess) return ctx_cuda(c_, e, "last-row readback");
        return EVSL_OK;
    }

    // Non-restart variant (ChebLanNr), called when the sum test of the Ritz values >= bar is
    // stable, when the slice looks empty, or when the basis is full (`full`): the candidates are
    // extracted as at a restart; if every one in the slice meets the locking tolerance (or the
    // basis is full) the converged ones become the result and the run ends, otherwise the same
    // basis keeps growing and the sum test starts over.
    int end_cycle_nr(bool full)
    {
        cudaEventRecord(e0_, c_->stream);
        const int k = k_;
        last_k_ = k;
        nrestart_++;
        int st = EVSL_OK;
        double *Yt = (double *)ctx_ws(c_, WS_LAN_Y, sizeof(double) * n_ * m_, &st);
        if (st) return st;
        Cands cd;
        EVSL_TRY(ritz_candidates(k, Yt, &cd));
        std::vector<int> conv;
        int unconv = 0;
        for (int cnd = 0; cnd < cd.ncand0; cnd++) {
            const double lj = cd.lam[cnd];
            const bool inside = (lj >= a_ - widen_) && ((right_closed_ || widen_ > 0) ? (lj <= b_ + widen_) : (lj < b_));
            if (!inside) continue;
            const double rj = std::sqrt(std::max(0.0, cd.res[cnd])) / normA_;
            if (rj <= tol_lock_) conv.push_back(cnd);
            else unconv++;
        }
        if (verbose_)
            fprintf(stderr, "[evsl] extraction %d: k=%d cand>=bar=%d converged=%zu unconverged=%d%s\n", nrestart_, k,
                    cd.ncand0, conv.size(), unconv, full ? " (basis full)" : "");
        if (unconv == 0 || full) {
            if ((int)conv.size() > cap_) {
                status_ = EVSL_ERR_CAPACITY;
                conv.resize(cap_);
            } else if (unconv > 0) {
                status_ = EVSL_ERR_NOCONV;
            }
            if (!conv.empty()) {
                int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * (size_t)(2 * (m_ + 1) + 8), &st);
                if (st) return st;
                EVSL_TRY(h2d(c_, idx, conv.data(), sizeof(int) * conv.size()));
                EVSL_TRY(gather_cols(c_, n_, (int)conv.size(), Yt, n_, idx, U_, n_));
                for (int cnd : conv) {
                    lam_l_.push_back(cd.lam[cnd]);
                    res_l_.push_back(std::sqrt(std::max(0.0, cd.res[cnd])) / normA_);
                }
                nlock_ = (int)conv.size();
            }
            done_ = true;
        } else {
            have_old_ = false;  // extend the same basis; the sum test starts over
            prev_nabove_ = 0;
        }
        cudaEventRecord(e1_, c_->stream);
        cudaEventSynchronize(e1_);
        t_restart_ += ev_ms(e0_, e1_) * 1e-3;
        return EVSL_OK;
    }

    // Restart: Ritz pairs of T_k, candidates theta >= bar, Rayleigh quotients with A, locking.
    int end_cycle()
    {
        cudaEventRecord(e0_, c_->stream);
        const int k = k_;
        last_k_ = k;
        nrestart_++;
        int st = EVSL_OK;
        double *Yt = (double *)ctx_ws(c_, WS_LAN_Y, sizeof(double) * n_ * m_, &st);
        if (st) return st;
        Cands cd;
        EVSL_TRY(ritz_candidates(k, Yt, &cd));
        int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * (size_t)(2 * (m_ + 1) + 8), &st);
        if (st) return st;
        const int ncand0 = cd.ncand0, sweeps = cd.sweeps;
        const double betak = cd.betak;
        const std::vector<double> &w = cd.w, &lamh = cd.lam, &resh = cd.res, &slast = cd.slast;
        const std::vector<int> &order = cd.order;
        int ncand = 0;
        const int nlock_before = nlock_;
        std::vector<int> lock_idx, tr_idx;
        std::vector<double> new_trtheta, new_trs, tr_res;
        if (ncand0 > 0) {
            for (int cnd = 0; cnd < ncand0; cnd++) {
                double lj = lamh[cnd];
                bool inside = (lj >= a_ - widen_) && ((right_closed_ || widen_ > 0) ? (lj <= b_ + widen_) : (lj < b_));
                if (!inside) continue;
                ncand++;
                double rj = std::sqrt(std::max(0.0, resh[cnd])) / normA_;
                if (rj <= tol_lock_) {
                    if (nlock_ + (int)lock_idx.size() >= cap_) {
                        status_ = EVSL_ERR_CAPACITY;
                        break;
                    }
                    lock_idx.push_back(cnd);
                    lam_l_.push_back(lj);
                    res_l_.push_back(rj);
                } else if ((int)tr_idx.size() < m_ / 2) {
                    // thick-restart set, largest Ritz values first, at most m/2 vectors
                    tr_res.push_back(rj);
                    tr_idx.push_back(cnd);
                    new_trtheta.push_back(w[order[cnd]]);
                    new_trs.push_back(betak * slast[cnd]);
                }
            }
            if (!lock_idx.empty()) {
                EVSL_TRY(h2d(c_, idx + (m_ + 1), lock_idx.data(), sizeof(int) * lock_idx.size()));
                EVSL_TRY(gather_cols(c_, n_, (int)lock_idx.size(), Yt, n_, idx + (m_ + 1), U_ + (int64_t)nlock_ * n_, n_));
                nlock_ += (int)lock_idx.size();
            }
        }
        if (status_ == EVSL_ERR_CAPACITY) return finish_run();
        const int ntr = (int)tr_idx.size();
        if (verbose_) {
            double rmin = 1e300;
            for (double r : tr_res) rmin = std::min(rmin, r);
            fprintf(stderr, "[evsl] restart %d: its=%d k=%d l=%d jacobi_sweeps=%d cand>=bar=%d in_slice=%d "
                            "locked+%d ntr=%d nlock=%d beta_k=%.3e min_unconverged_res=%.3e\n",
                    nrestart_, its_, k, l_, sweeps, ncand0, ncand, (int)lock_idx.size(), ntr, nlock_, betak,
                    tr_res.empty() ? 0.0 : rmin);
        }
        if (ncand == 0) nocand_++; else nocand_ = 0;
        if (ncand > 0 && nlock_ == nlock_before) stall_++; else stall_ = 0;
        if (mixed_ && stall_ >= 2 && tol_lock_ < MIXED_TOL_LOCK_MAX) {
            // candidates in the slice that no longer improve: the FP32 filter's accuracy floor
            // lies above the locking level, so relax it (the FP64 polish restores tol)
            tol_lock_ = std::min(MIXED_TOL_LOCK_MAX, 10.0 * tol_lock_);
            widen_ = tol_lock_ * normA_;
            stall_ = 0;
        }
        bool refined = false;
        if (stall_ >= 2 && nrefine_ < 2 && ntr > 0 && nlock_ + ntr <= cap_) {
            // stagnation: Rayleigh-Ritz with A over the locked set and the stuck candidates
            EVSL_TRY(h2d(c_, idx, tr_idx.data(), sizeof(int) * ntr));
            EVSL_TRY(gather_cols(c_, n_, ntr, Yt, n_, idx, U_ + (int64_t)nlock_ * n_, n_));
            int kept = 0;
            EVSL_TRY(refine_locked(nlock_ + ntr, &kept));
            nlock_ = kept;
            nrefine_++;
            stall_ = 0;
            nocand_ = 1;
            refined = true;
        }
        cudaEventRecord(e1_, c_->stream);
        cudaEventSynchronize(e1_);
        t_restart_ += ev_ms(e0_, e1_) * 1e-3;
        if (nocand_ >= 2) return finish_run();
        if (its_ > maxit_) {
            status_ = EVSL_ERR_NOCONV;
            return finish_run();
        }
        if (ncand == 0 || refined) {
            l_ = 0;
            EVSL_TRY(fresh_vector(fresh_index_++, Q_, nlock_, 0));
        } else {
            if (ntr != k) EVSL_TRY(d2d(c_, Q_ + (int64_t)ntr * n_, Q_ + (int64_t)k * n_, sizeof(double) * n_));
            if (ntr > 0) {
                EVSL_TRY(h2d(c_, idx, tr_idx.data(), sizeof(int) * ntr));
                EVSL_TRY(gather_cols(c_, n_, ntr, Yt, n_, idx, Q_, n_));
            }
            trtheta_ = new_trtheta;
            trs_ = new_trs;
            l_ = ntr;
            if (l_ == 0) {
                // continue from q_{k+1}, re-orthogonalised against the new locked vectors
                EVSL_TRY(coldot(c_, n_, 1, Q_, n_, Q_, n_, sc_ + TMP));
                double b2 = 0;
                EVSL_TRY(d2h(c_, &b2, sc_ + TMP, sizeof(double)));
                double nrm2;
                EVSL_TRY(reorth(Q_, 0, b2, &nrm2));
                EVSL_TRY(scale_vec(c_, n_, Q_, 1.0 / std::sqrt(nrm2), nullptr));
            }
        }
        begin_cycle();
        return EVSL_OK;
    }

    int finish_run()
    {
        done_ = true;
        return EVSL_OK;
    }

    bool in_slice(double t) const { return t >= a_ && (right_closed_ ? t <= b_ : t < b_); }

    // After orthonormalize kept k < want columns of X: fresh seeded vectors fill columns
    // k..want-1 and the block is orthonormalised again (Tmp: n x want scratch).
    int refill_block(double *X, int k, int want, double *Tmp, int *kout)
    {
        int kk = k;
        for (int tries = 0; tries < 3 && kk < want; tries++) {
            for (int j = kk; j < want; j++)
                EVSL_TRY(fill_uniform_f64(c_, n_, o_.seed, SM_STREAM_LANCZOS, fresh_index_++, X + (int64_t)j * n_));
            EVSL_TRY(orthonormalize(X, want, Tmp, &kk));
        }
        *kout = kk;
        return EVSL_OK;
    }

    // FP64 recovery after an FP32-filter run: restarted block Krylov iteration with the FP64
    // filter.  The start block V0 = orth[U, G] holds the pairs the FP32 phase locked and g guard
    // vectors (the leading vectors of its last Krylov basis: orthogonal to U and dominated by
    // the largest rho below bar, i.e. the eigenvectors just outside the slice).  Each cycle
    // builds Q = [V0, V1, V2] with V_{j+1} = orth((I - Q Q^T) rho(Ahat) V_j) and keeps
    // R = rho(Ahat) Q.  H = Q^T R gives the Ritz values mu of rho on span(Q); the Ritz vectors
    // with mu >= 0.9 bar and ||rho y - mu y|| <= 1e-3 |mu| (from R^T R) span a nearly invariant
    // subspace, and a Rayleigh-Ritz step with A on it gives the eigenpair estimates; directions
    // that have not converged stay out of that projection, where they would make spurious
    // Ritz values inside the slice.  The next cycle starts from the k0 Ritz vectors of rho with
    // the largest mu.  The error of an in-slice eigenvector along the eigenvectors just outside
    // the slice, where rho is close to bar on both sides, falls much faster in the Krylov space
    // than under plain subspace iteration.  The cycles stop when every estimate in the slice
    // meets tol and no Ritz value >= bar is left unconverged; the converged in-slice pairs are
    // the result (EVSL_ERR_NOCONV if some never met tol, EVSL_ERR_CAPACITY if more than cap did).
    int polish()
    {
        const int p = nlock_;
        if (p == 0) return EVSL_OK;
        const int g = std::min(std::max(16, p / 4), 256);
        const int k0 = (int)std::min<int64_t>(p + g, n_);
        const int nb = POLISH_BLOCKS;
        const int64_t kmax = std::min<int64_t>((int64_t)nb * k0, n_);
        const int nc = std::min(k0, 64);
        int st = EVSL_OK;
        double *Q = (double *)ctx_ws(c_, WS_POL_V, sizeof(double) * n_ * kmax, &st);
        if (st) return st;
        double *R = (double *)ctx_ws(c_, WS_POL_W, sizeof(double) * n_ * kmax, &st);
        if (st) return st;
        double *Ys = (double *)ctx_ws(c_, WS_POL_Y, sizeof(double) * n_ * k0, &st);
        if (st) return st;
        double *Out = (double *)ctx_ws(c_, WS_LAN_Y, sizeof(double) * n_ * std::max(m_, k0), &st);
        if (st) return st;
        double *B = (double *)ctx_ws(c_, WS_POL_B, sizeof(double) * n_ * 2 * nc, &st);
        if (st) return st;
        const int kq = std::min(last_k_, k0 - p);
        EVSL_TRY(d2d(c_, Q, U_, sizeof(double) * n_ * p));
        if (kq > 0) EVSL_TRY(d2d(c_, Q + (int64_t)p * n_, Q_, sizeof(double) * n_ * kq));
        for (int j = p + kq; j < k0; j++)
            EVSL_TRY(fill_uniform_f64(c_, n_, o_.seed, SM_STREAM_LANCZOS, fresh_index_++, Q + (int64_t)j * n_));
        int kb0 = 0;
        EVSL_TRY(orthonormalize(Q, k0, Ys, &kb0));
        std::vector<double> th, r2;
        double best_rmax = 0.0;
        for (int cyc = 0; cyc < POLISH_CYCLES && kb0 > 0; cyc++) {
            // block Krylov basis Q[:, :Kt] and R = rho(Ahat) Q
            int off = 0, kb = kb0, Kt = 0;
            for (int j = 0; j < nb; j++) {
                for (int j0 = 0; j0 < kb; j0 += nc) {
                    const int m = std::min(nc, kb - j0);
                    const int64_t o = (int64_t)(off + j0) * n_;
                    EVSL_TRY(filter_apply_dev(c_, pol_, m, Q + o, R + o, EVSL_FP64, B, B + (int64_t)m * n_, nullptr));
                }
                Kt = off + kb;
                if (j + 1 == nb) break;
                const int kn = (int)std::min<int64_t>(kb, kmax - Kt);
                if (kn <= 0) break;
                double *Nb = Q + (int64_t)Kt * n_;
                EVSL_TRY(d2d(c_, Nb, R + (int64_t)off * n_, sizeof(double) * n_ * kn));
                double *G = (double *)ctx_ws(c_, WS_LAN_G, sizeof(double) * (size_t)Kt * kn, &st);
                if (st) return st;
                for (int pass = 0; pass < 2; pass++) {
                    EVSL_TRY(gemm_tn(c_, n_, Kt, kn, Q, n_, Nb, n_, G, Kt));
                    EVSL_TRY(gemm_nn_sub(c_, n_, kn, Kt, Q, n_, G, Kt, Nb, n_));
                }
                int knew = 0;
                EVSL_TRY(orthonormalize(Nb, kn, Ys, &knew));
                if (knew == 0) break;
                off = Kt;
                kb = knew;
            }
            // Ritz values of rho on span(Q): H = Q^T R; residuals in rho from R^T R
            double *G = (double *)ctx_ws(c_, WS_LAN_G, sizeof(double) * (size_t)Kt * Kt, &st);
            if (st) return st;
            EVSL_TRY(gemm_tn(c_, n_, Kt, Kt, Q, n_, R, n_, G, Kt));
            std::vector<double> Gh((size_t)Kt * Kt), mu(Kt);
            EVSL_TRY(d2h(c_, Gh.data(), G, sizeof(double) * Gh.size()));
            symmetrize(Gh, Kt);
            const int M = std::max(2, Kt + (Kt & 1));
            double *Vj = (double *)ctx_ws(c_, WS_LAN_T, sizeof(double) * (size_t)M * M, &st);
            if (st) return st;
            int ldv = 0, sweeps = 0;
            EVSL_TRY(jacobi_eig(c_, Kt, Gh.data(), mu.data(), Vj, &ldv, &sweeps));
            EVSL_TRY(gemm_tn(c_, n_, Kt, Kt, R, n_, R, n_, G, Kt));
            std::vector<int> order(Kt);
            std::iota(order.begin(), order.end(), 0);
            std::sort(order.begin(), order.end(), [&](int x, int y) { return mu[x] > mu[y]; });
            int ncand = 0;
            while (ncand < Kt && mu[order[ncand]] >= POLISH_SELECT * bar_) ncand++;
            std::vector<int> sel;
            bool pending = false;  // a Ritz value >= bar whose vector has not converged yet
            double *Sd = (double *)ctx_ws(c_, WS_LAN_S, sizeof(double) * (size_t)M * M, &st);
            if (st) return st;
            int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * ((size_t)Kt + 8), &st);
            if (st) return st;
            // the restart block's coefficients (the Rayleigh-Ritz step below reuses Vj's memory)
            const int kr = std::min(k0, Kt);
            double *Stop = (double *)ctx_ws(c_, WS_POL_R, sizeof(double) * (size_t)Kt * kr, &st);
            if (st) return st;
            EVSL_TRY(h2d(c_, idx, order.data(), sizeof(int) * kr));
            EVSL_TRY(gather_cols(c_, Kt, kr, Vj, ldv, idx, Stop, Kt));
            if (ncand > 0) {
                double *T = (double *)ctx_ws(c_, WS_POL_S, sizeof(double) * ((size_t)Kt * ncand + ncand + 8), &st);
                if (st) return st;
                double *qd = T + (size_t)Kt * ncand;
                EVSL_TRY(h2d(c_, idx, order.data(), sizeof(int) * ncand));
                EVSL_TRY(gather_cols(c_, Kt, ncand, Vj, ldv, idx, Sd, Kt));
                EVSL_TRY(gemm_nn(c_, Kt, ncand, Kt, G, Kt, Sd, Kt, T, Kt));
                EVSL_TRY(coldot(c_, Kt, ncand, Sd, Kt, T, Kt, qd));
                std::vector<double> q(ncand);
                EVSL_TRY(d2h(c_, q.data(), qd, sizeof(double) * ncand));
                for (int t = 0; t < ncand; t++) {
                    const double mj = mu[order[t]];
                    const double rr = std::sqrt(std::max(0.0, q[t] - mj * mj));
                    if (rr <= POLISH_RHO_RES * std::fabs(mj) && (int)sel.size() < k0) sel.push_back(order[t]);
                    else if (mj >= bar_) pending = true;
                }
            }
            const int ks = (int)sel.size();
            th.clear();
            r2.clear();
            bool ok = !pending;
            int nin = 0;
            double rmax = 0.0;
            if (ks > 0) {
                EVSL_TRY(h2d(c_, idx, sel.data(), sizeof(int) * ks));
                EVSL_TRY(gather_cols(c_, Kt, ks, Vj, ldv, idx, Sd, Kt));
                EVSL_TRY(gemm_nn(c_, n_, ks, Kt, Q, n_, Sd, Kt, Ys, n_));
                int sw2 = 0;
                EVSL_TRY(rayleigh_ritz(Ys, ks, Out, th, r2, &sw2));
                for (int j = 0; j < ks; j++)
                    if (in_slice(th[j])) {
                        const double rj = std::sqrt(std::max(0.0, r2[j])) / normA_;
                        nin++;
                        rmax = std::max(rmax, rj);
                        if (rj > tol_) ok = false;
                    }
            }
            if (verbose_)
                fprintf(stderr, "[evsl] polish cycle %d: basis=%d selected=%d pending=%d in_slice=%d max_res=%.3e\n",
                        cyc, Kt, ks, (int)pending, nin, rmax);
            if (ok || cyc + 1 == POLISH_CYCLES) break;
            // a cycle that made the worst residual ten times larger has picked up mixtures
            // of eigenvectors; more cycles would not recover, the caller falls back to FP64
            if (cyc > 0 && rmax > 10.0 * best_rmax) break;
            best_rmax = cyc == 0 ? rmax : std::min(best_rmax, rmax);
            // restart from the k0 Ritz vectors of rho with the largest mu
            kb0 = kr;
            EVSL_TRY(gemm_nn(c_, n_, kb0, Kt, Q, n_, Stop, Kt, Ys, n_));
            EVSL_TRY(d2d(c_, Q, Ys, sizeof(double) * n_ * kb0));
        }
        std::vector<int> keep;
        lam_l_.clear();
        res_l_.clear();
        bool all = true;
        int nconv = 0;
        for (int j = 0; j < (int)th.size(); j++) {
            if (!in_slice(th[j])) continue;
            const double rj = std::sqrt(std::max(0.0, r2[j])) / normA_;
            if (rj > tol_) {
                all = false;
                continue;
            }
            nconv++;
            if ((int)keep.size() < cap_) {
                keep.push_back(j);
                lam_l_.push_back(th[j]);
                res_l_.push_back(rj);
            }
        }
        if (!keep.empty()) {
            int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * (keep.size() + 8), &st);
            if (st) return st;
            EVSL_TRY(h2d(c_, idx, keep.data(), sizeof(int) * keep.size()));
            EVSL_TRY(gather_cols(c_, n_, (int)keep.size(), Out, n_, idx, U_, n_));
        }
        nlock_ = (int)keep.size();
        if (nconv > cap_) status_ = EVSL_ERR_CAPACITY;
        else if (!all && status_ == EVSL_OK) status_ = EVSL_ERR_NOCONV;
        return EVSL_OK;
    }

    // The FP32-filter run's fallback: a fresh FP64 thick-restart run of the same slice (its
    // basis memory replaces this run's Krylov basis, which is no longer needed); its pairs,
    // status and step counts become this run's.
    int resolve_fp64()
    {
        if (verbose_) fprintf(stderr, "[evsl] FP64 polish left pairs above tol: the slice is solved again in FP64\n");
        ctx_free(c_, Q_, sizeof(double) * n_ * (m_ + 1));
        Q_ = nullptr;
        evsl_lan_opts o = o_;
        o.prec = EVSL_FP64;
        SliceSolver S(c_, a_, b_, pol_, o, m_, cap_, right_closed_);
        EVSL_TRY(S.init());
        int st = EVSL_OK;
        double *y = (double *)ctx_ws(c_, WS_LAN_VEC, sizeof(double) * n_ * 3, &st);
        if (st) return st;
        while (!S.done()) {
            cudaEventRecord(e0_, c_->stream);
            EVSL_TRY(filter_apply_dev(c_, pol_, 1, S.input(), y, EVSL_FP64, y + n_, y + 2 * n_, nullptr));
            cudaEventRecord(e1_, c_->stream);
            cudaEventSynchronize(e1_);
            EVSL_TRY(S.consume(y, ev_ms(e0_, e1_) * 1e-3));
        }
        nlock_ = S.nlock_;
        lam_l_ = S.lam_l_;
        res_l_ = S.res_l_;
        status_ = S.status_;
        if (nlock_ > 0) EVSL_TRY(d2d(c_, U_, S.U_, sizeof(double) * n_ * nlock_));
        its_ += S.its_;
        nmv_ += S.nmv_;
        npass_ += S.npass_;
        nrestart_ += S.nrestart_;
        t_filter_ += S.t_filter_;
        t_orth_ += S.t_orth_;
        t_restart_ += S.t_restart_;
        return EVSL_OK;
    }

    // In place: the k columns of W become an orthonormal basis of their span (*kr columns).
    // Columns are scaled to unit norm, then two passes of W <- W S diag(s)^(-1/2) with
    // W^T W = S diag(s) S^T; the first pass drops directions with s <= 1e-12 max(s), i.e.
    // columns that are (to about 1e-6) combinations of the others.  Tmp: n x k scratch.
    int orthonormalize(double *W, int k, double *Tmp, int *kr)
    {
        int st = EVSL_OK;
        double *sd = (double *)ctx_ws(c_, WS_POL_S, sizeof(double) * ((size_t)k + 8), &st);
        if (st) return st;
        std::vector<double> nr(k), scl;
        EVSL_TRY(coldot(c_, n_, k, W, n_, W, n_, sd));
        EVSL_TRY(d2h(c_, nr.data(), sd, sizeof(double) * k));
        for (int j = 0; j < k; j++) nr[j] = nr[j] > 0.0 ? 1.0 / std::sqrt(nr[j]) : 0.0;
        EVSL_TRY(h2d(c_, sd, nr.data(), sizeof(double) * k));
        EVSL_TRY(colscale(c_, n_, k, W, sd));
        int kk = k;
        for (int pass = 0; pass < 2 && kk > 0; pass++) {
            double *G = (double *)ctx_ws(c_, WS_LAN_G, sizeof(double) * (size_t)kk * kk, &st);
            if (st) return st;
            EVSL_TRY(gemm_tn(c_, n_, kk, kk, W, n_, W, n_, G, kk));
            std::vector<double> Gh((size_t)kk * kk), sv(kk);
            EVSL_TRY(d2h(c_, Gh.data(), G, sizeof(double) * Gh.size()));
            symmetrize(Gh, kk);
            const int M = std::max(2, kk + (kk & 1));
            double *Vj = (double *)ctx_ws(c_, WS_LAN_T, sizeof(double) * (size_t)M * M, &st);
            if (st) return st;
            int ldv = 0, sweeps = 0;
            EVSL_TRY(jacobi_eig(c_, kk, Gh.data(), sv.data(), Vj, &ldv, &sweeps));
            double smax = 0.0;
            for (double v : sv) smax = std::max(smax, v);
            std::vector<int> kd;
            scl.clear();
            for (int j = 0; j < kk; j++)
                if (sv[j] > 1e-12 * smax) {
                    kd.push_back(j);
                    scl.push_back(1.0 / std::sqrt(sv[j]));
                }
            const int nk = (int)kd.size();
            if (nk == 0) {
                kk = 0;
                break;
            }
            double *Sd = (double *)ctx_ws(c_, WS_LAN_S, sizeof(double) * (size_t)M * M, &st);
            if (st) return st;
            int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * ((size_t)nk + 8), &st);
            if (st) return st;
            EVSL_TRY(h2d(c_, idx, kd.data(), sizeof(int) * nk));
            EVSL_TRY(gather_cols(c_, kk, nk, Vj, ldv, idx, Sd, kk));
            EVSL_TRY(h2d(c_, sd, scl.data(), sizeof(double) * nk));
            EVSL_TRY(colscale(c_, kk, nk, Sd, sd));
            EVSL_TRY(gemm_nn(c_, n_, nk, kk, W, n_, Sd, kk, Tmp, n_));
            EVSL_TRY(d2d(c_, W, Tmp, sizeof(double) * n_ * nk));
            kk = nk;
        }
        *kr = kk;
        return EVSL_OK;
    }

    static void symmetrize(std::vector<double> &Gh, int k)
    {
        for (int j = 0; j < k; j++)
            for (int i = 0; i < j; i++) {
                double v = 0.5 * (Gh[(size_t)j * k + i] + Gh[(size_t)i * k + j]);
                Gh[(size_t)j * k + i] = v;
                Gh[(size_t)i * k + j] = v;
            }
    }

    // Rayleigh-Ritz with A over the k orthonormal columns of Wb: Wb^T A Wb = S diag(th) S^T
    // with th ascending, Out = Wb S (Out must not alias Wb), r2[j] = ||A out_j - th_j out_j||^2.
    int rayleigh_ritz(const double *Wb, int k, double *Out, std::vector<double> &th,
                      std::vector<double> &r2, int *sweeps_out)
    {
        int st = EVSL_OK;
        const int zc = std::min(k, 128);
        double *Z = (double *)ctx_ws(c_, WS_LAN_Z, sizeof(double) * n_ * zc, &st);
        if (st) return st;
        double *G = (double *)ctx_ws(c_, WS_LAN_G, sizeof(double) * (size_t)k * k, &st);
        if (st) return st;
        for (int j0 = 0; j0 < k; j0 += zc) {
            int nc = std::min(zc, k - j0);
            EVSL_TRY(spmv_f64(c_, nc, Wb + (int64_t)j0 * n_, Z));
            EVSL_TRY(gemm_tn(c_, n_, k, nc, Wb, n_, Z, n_, G + (int64_t)j0 * k, k));
        }
        std::vector<double> Gh((size_t)k * k), w(k);
        EVSL_TRY(d2h(c_, Gh.data(), G, sizeof(double) * Gh.size()));
        symmetrize(Gh, k);
        const int M = std::max(2, k + (k & 1));
        double *Vj = (double *)ctx_ws(c_, WS_LAN_T, sizeof(double) * (size_t)M * M, &st);
        if (st) return st;
        int ldv = 0, sweeps = 0;
        EVSL_TRY(jacobi_eig(c_, k, Gh.data(), w.data(), Vj, &ldv, &sweeps));
        double *Sd = (double *)ctx_ws(c_, WS_LAN_S, sizeof(double) * (size_t)M * M, &st);
        if (st) return st;
        std::vector<int> order(k);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] < w[y]; });
        int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * (size_t)(2 * k + 8), &st);
        if (st) return st;
        EVSL_TRY(h2d(c_, idx, order.data(), sizeof(int) * k));
        EVSL_TRY(gather_cols(c_, k, k, Vj, ldv, idx, Sd, k));
        EVSL_TRY(gemm_nn(c_, n_, k, k, Wb, n_, Sd, k, Out, n_));
        th.assign(k, 0.0);
        r2.assign(k, 0.0);
        for (int j = 0; j < k; j++) th[j] = w[order[j]];
        double *lamd = (double *)ctx_ws(c_, WS_KPM_PART, sizeof(double) * 2 * (size_t)k, &st);
        if (st) return st;
        EVSL_TRY(h2d(c_, lamd, th.data(), sizeof(double) * k));
        for (int j0 = 0; j0 < k; j0 += zc) {
            int nc = std::min(zc, k - j0);
            EVSL_TRY(spmv_f64(c_, nc, Out + (int64_t)j0 * n_, Z));
            EVSL_TRY(colres2(c_, n_, nc, Z, Out + (int64_t)j0 * n_, n_, lamd + j0, lamd + k + j0));
        }
        EVSL_TRY(d2h(c_, r2.data(), lamd + k, sizeof(double) * k));
        *sweeps_out = sweeps;
        return EVSL_OK;
    }

    // Rayleigh-Ritz refinement with A over W = U[:, :p] (orthonormal columns): the Ritz
    // vectors with theta in the (possibly widened) slice and ||A w - theta w|| <= tol_lock ||A||
    // replace the locked set, in ascending theta.
    int refine_locked(int p, int *kept_out)
    {
        int st = EVSL_OK;
        double *Yt = (double *)ctx_ws(c_, WS_LAN_Y, sizeof(double) * n_ * std::max(m_, p), &st);
        if (st) return st;
        std::vector<double> th, r2;
        int sweeps = 0;
        EVSL_TRY(rayleigh_ritz(U_, p, Yt, th, r2, &sweeps));
        std::vector<int> keep;
        lam_l_.clear();
        res_l_.clear();
        for (int j = 0; j < p; j++) {
            bool inside = (th[j] >= a_ - widen_) &&
                          ((right_closed_ || widen_ > 0) ? (th[j] <= b_ + widen_) : (th[j] < b_));
            double rj = std::sqrt(std::max(0.0, r2[j])) / normA_;
            if (inside && rj <= tol_lock_ && (int)keep.size() < cap_) {
                keep.push_back(j);
                lam_l_.push_back(th[j]);
                res_l_.push_back(rj);
            }
        }
        if (!keep.empty()) {
            int *idx = (int *)ctx_ws(c_, WS_LAN_IDX, sizeof(int) * (size_t)(2 * p + 8), &st);
            if (st) return st;
            EVSL_TRY(h2d(c_, idx + p, keep.data(), sizeof(int) * keep.size()));
            EVSL_TRY(gather_cols(c_, n_, (int)keep.size(), Yt, n_, idx + p, U_, n_));
        }
        if (verbose_) fprintf(stderr, "[evsl] refinement: p=%d kept=%zu sweeps=%d\n", p, keep.size(), sweeps);
        *kept_out = (int)keep.size();
        return EVSL_OK;
    }

    evsl_ctx *c_;
    int64_t n_;
    double a_, b_;
    const evsl_polfilt *pol_;
    evsl_lan_opts o_;
    int m_ = 0, cap_ = 0, maxit_ = 0, ncycle_ = 10;
    bool right_closed_ = true, nonrestart_ = false, verbose_ = false, mixed_ = false;
    double tol_ = 1e-8, tau1_ = 1e-10, bar_ = 0.0, normA_ = 1.0, tol_lock_ = 1e-8, widen_ = 0.0;
    double *U_ = nullptr, *Q_ = nullptr, *sc_ = nullptr, *h_ = nullptr;
    size_t nsc_ = 0;
    std::vector<double> T_, trtheta_, trs_, lam_l_, res_l_;
    int nlock_ = 0, l_ = 0, k_ = 0, i_ = 0, lstart_ = 0, its_ = 0, nrestart_ = 0, nocand_ = 0;
    int stall_ = 0, nrefine_ = 0, prev_nabove_ = 0, last_k_ = 0;
    bool tr_pending_ = false, have_old_ = false, done_ = false;
    double t_old_ = 0.0;
    uint64_t fresh_index_ = 0;
    int status_ = EVSL_OK;
    int64_t nmv_ = 0, npass_ = 0;
    double t_filter_ = 0, t_orth_ = 0, t_restart_ = 0;
    cudaEvent_t e0_ = nullptr, e1_ = nullptr, e2_ = nullptr;
};

int status_message(evsl_ctx *c, int st, int cap, int maxit)
{
    if (st == EVSL_ERR_CAPACITY) return ctx_fail(c, st, "more than cap=%d eigenpairs converged", cap);
    if (st == EVSL_ERR_NOCONV)
        return ctx_fail(c, st, "some eigenpairs of the slice did not reach tol (maxit=%d Lanczos steps, or "
                               "the FP64 polish cycles after an FP32 filter ran out)", maxit);
    return st;
}

}  // namespace

// ------------------------------------------------------------------------------------------
int drv_chebLanTr(evsl_ctx *c, double a, double b, const evsl_polfilt *pol,
                  const evsl_lan_opts *o, int cap, int *nev, double *lam, double *Y, double *res,
                  evsl_stats *st, bool nonrestart)
{
    cudaEvent_t ta, tb, fa, fb;
    cudaEventCreate(&ta);
    cudaEventCreate(&tb);
    cudaEventCreate(&fa);
    cudaEventCreate(&fb);
    cudaEventRecord(ta, c->stream);
    int rc = EVSL_OK;
    {
        SliceSolver S(c, a, b, pol, *o, o->m, cap, o->right_closed != 0, nonrestart);
        rc = S.init();
        const int64_t n = c->A.n;
        double *y = nullptr, *B0 = nullptr, *B1 = nullptr;
        float *fbuf = nullptr;
        if (rc == EVSL_OK) {
            y = (double *)ctx_ws(c, WS_LAN_VEC, sizeof(double) * n * 3, &rc);
            if (o->prec == EVSL_FP32 && rc == EVSL_OK)
                fbuf = (float *)ctx_ws(c, WS_F32_X, sizeof(float) * 4 * n, &rc);
        }
        if (y) {
            B0 = y + n;
            B1 = y + 2 * n;
        }
        while (rc == EVSL_OK && !S.done()) {
            cudaEventRecord(fa, c->stream);
            rc = filter_apply_dev(c, pol, 1, S.input(), y, o->prec, B0, B1, fbuf);
            if (rc != EVSL_OK) break;
            cudaEventRecord(fb, c->stream);
            cudaEventSynchronize(fb);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, fa, fb);
            rc = S.consume(y, ms * 1e-3);
        }
        if (rc == EVSL_OK) {
            cudaEventRecord(tb, c->stream);
            cudaEventSynchronize(tb);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ta, tb);
            rc = S.finish(nev, lam, res, Y, st, ms * 1e-3);
            if (rc == EVSL_OK)
                rc = status_message(c, S.status(), cap, nonrestart ? o->m : (o->maxit > 0 ? o->maxit : 20 * o->m));
        }
    }
    cudaEventDestroy(ta);
    cudaEventDestroy(tb);
    cudaEventDestroy(fa);
    cudaEventDestroy(fb);
    return rc;
}

// ------------------------------------------------------------------------------------------
// Incremental lockstep batch: slice jobs join (evsl_batch_add) and leave (when finished) between
// steps; every step applies all active jobs' filters in one multi-slice pass per degree.
struct evsl_batch {
    evsl_ctx *c = nullptr;
    evsl_lan_opts o{};
    std::vector<std::unique_ptr<SliceSolver>> solvers;
    std::vector<evsl_slice_job *> jobs;
    std::vector<std::chrono::steady_clock::time_point> t0;
    cudaEvent_t fa = nullptr, fb = nullptr;
};

int batch_create(evsl_ctx *c, const evsl_lan_opts *o, evsl_batch **out)
{
    evsl_batch *bt = new evsl_batch();
    bt->c = c;
    bt->o = *o;
    cudaEventCreate(&bt->fa);
    cudaEventCreate(&bt->fb);
    c->batches.push_back(bt);
    *out = bt;
    return EVSL_OK;
}

void batch_destroy(evsl_batch *bt)
{
    if (!bt) return;
    auto &v = bt->c->batches;
    v.erase(std::remove(v.begin(), v.end(), bt), v.end());
    cudaStreamSynchronize(bt->c->stream);
    bt->solvers.clear();
    if (bt->fa) cudaEventDestroy(bt->fa);
    if (bt->fb) cudaEventDestroy(bt->fb);
    delete bt;
}

// Device bytes the shared workspaces still have to grow by so that a step (batched filter) and
// a restart / refinement of any active job fit: admission reserves them before accepting a job.
static size_t workspace_growth(evsl_ctx *c, const evsl_batch *bt, const evsl_slice_job *job)
{
    const size_t n = (size_t)c->A.n;
    size_t na = bt->solvers.size() + 1;
    int mmax = job->m, capmax = job->cap, degmax = job->pol->deg;
    for (const evsl_slice_job *J : bt->jobs) {
        mmax = std::max(mmax, J->m);
        capmax = std::max(capmax, J->cap);
        degmax = std::max(degmax, J->pol->deg);
    }
    const size_t big = std::max<size_t>(mmax, 2 * (size_t)capmax);
    size_t need = 0;
    auto want = [&](int slot, size_t bytes) {
        size_t have = (c->ws_bytes.size() > (size_t)slot) ? c->ws_bytes[slot] : 0;
        if (bytes > have) need += bytes - have;
    };
    want(WS_LAN_VEC, sizeof(double) * 2 * n * na);
    want(WS_W2, sizeof(double) * 2 * n * na);
    want(WS_W0, sizeof(double) * std::max<size_t>(n * na, 2 * n * 128));
    want(WS_W1, sizeof(double) * n * na);
    if (bt->o.prec == EVSL_FP32) want(WS_F32_X, sizeof(float) * 4 * n * na);
    want(WS_KPM_PART, sizeof(double) * ((size_t)(degmax + 1) * na + 2 * big + 64));
    want(WS_LAN_Y, sizeof(double) * n * big);
    want(WS_LAN_Z, sizeof(double) * n * 128);
    want(WS_LAN_T, sizeof(double) * (big + 2) * (big + 2));
    want(WS_LAN_S, sizeof(double) * (big + 2) * (big + 2));
    want(WS_LAN_G, sizeof(double) * big * big);
    want(WS_PARTIAL, sizeof(double) * ((n + 2047) / 2048 + 1) * (size_t)(capmax + mmax + 1 + 64));
    return need;
}

int batch_add(evsl_batch *bt, evsl_slice_job *job)
{
    evsl_ctx *c = bt->c;
    job->status = EVSL_OK;
    *job->nev = 0;
    const size_t need = workspace_growth(c, bt, job);
    const size_t bases = sizeof(double) * (size_t)c->A.n * ((size_t)job->cap + job->m + 1);
    if (c->budget && c->used + need + bases > c->budget)
        return ctx_fail(c, EVSL_ERR_NOMEM, "batch_add: HBM budget has no room for the job (%zu + %zu + %zu > %zu bytes)",
                        c->used, bases, need, c->budget);
    const size_t dcap = dev_budget_bytes(c->device), dused = dev_used_bytes(c->device);
    if (dcap && dused + need + bases > dcap)
        return ctx_fail(c, EVSL_ERR_NOMEM,
                        "batch_add: device HBM budget has no room for the job (%zu + %zu + %zu > %zu bytes)", dused,
                        bases, need, dcap);
    std::unique_ptr<SliceSolver> s(new SliceSolver(c, job->a, job->b, job->pol, bt->o, job->m, job->cap,
                                                   job->right_closed != 0));
    int rc = s->init();
    if (rc != EVSL_OK) return rc;  // the solver's memory is released by its destructor
    bt->solvers.push_back(std::move(s));
    bt->jobs.push_back(job);
    bt->t0.push_back(std::chrono::steady_clock::now());
    return EVSL_OK;
}

int batch_step(evsl_batch *bt, int *nactive, int *nfinished)
{
    evsl_ctx *c = bt->c;
    const int64_t n = c->A.n;
    int finished = 0;
    const int na = (int)bt->solvers.size();
    if (na > 0) {
        int rc = EVSL_OK;
        double *Xb = (double *)ctx_ws(c, WS_LAN_VEC, sizeof(double) * n * 2 * na, &rc);
        if (rc) return rc;
        double *Yb = Xb + n * na;
        std::vector<evsl_polfilt> pols(na);
        for (int t = 0; t < na; t++) {
            pols[t] = *bt->solvers[t]->pol();
            cudaError_t e = cudaMemcpyAsync(Xb + (int64_t)t * n, bt->solvers[t]->input(), sizeof(double) * n,
                                            cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) return ctx_cuda(c, e, "batch gather");
        }
        cudaEventRecord(bt->fa, c->stream);
        if (na == 1) {
            double *B = nullptr;
            float *fbuf = nullptr;
            B = (double *)ctx_ws(c, WS_W0, sizeof(double) * n * 2, &rc);
            if (rc) return rc;
            if (bt->o.prec == EVSL_FP32) {
                fbuf = (float *)ctx_ws(c, WS_F32_X, sizeof(float) * 4 * n, &rc);
                if (rc) return rc;
            }
            EVSL_TRY(filter_apply_dev(c, &pols[0], 1, Xb, Yb, bt->o.prec, B, B + n, fbuf));
        } else {
            EVSL_TRY(filter_apply_multi_dev(c, na, pols.data(), Xb, Yb, bt->o.prec));
        }
        cudaEventRecord(bt->fb, c->stream);
        cudaEventSynchronize(bt->fb);
        const double tf = ev_ms(bt->fa, bt->fb) * 1e-3;
        for (int t = 0; t < na; t++) EVSL_TRY(bt->solvers[t]->consume(Yb + (int64_t)t * n, tf));
        // retire finished jobs: write their outputs and release their bases
        for (int t = na - 1; t >= 0; t--) {
            if (!bt->solvers[t]->done()) continue;
            evsl_slice_job *J = bt->jobs[t];
            double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - bt->t0[t]).count();
            EVSL_TRY(bt->solvers[t]->finish(J->nev, J->lam, J->res, J->Y, J->stats, secs));
            J->status = bt->solvers[t]->status();
            bt->solvers.erase(bt->solvers.begin() + t);
            bt->jobs.erase(bt->jobs.begin() + t);
            bt->t0.erase(bt->t0.begin() + t);
            finished++;
        }
    }
    if (nactive) *nactive = (int)bt->solvers.size();
    if (nfinished) *nfinished = finished;
    return EVSL_OK;
}

evsl_ctx *batch_ctx(evsl_batch *bt) { return bt->c; }

int drv_chebSI(evsl_ctx *c, double a, double b, const evsl_polfilt *pol, const evsl_lan_opts *o, int cap,
               int *nev, double *lam, double *Y, double *res, evsl_stats *st)
{
    cudaEvent_t ta, tb;
    cudaEventCreate(&ta);
    cudaEventCreate(&tb);
    cudaEventRecord(ta, c->stream);
    int rc = EVSL_OK;
    {
        SliceSolver S(c, a, b, pol, *o, o->m, cap, o->right_closed != 0);
        rc = S.init();
        if (rc == EVSL_OK) rc = S.run_si(o->maxit > 0 ? o->maxit : 100);
        if (rc == EVSL_OK) {
            cudaEventRecord(tb, c->stream);
            cudaEventSynchronize(tb);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ta, tb);
            rc = S.finish(nev, lam, res, Y, st, ms * 1e-3);
            if (rc == EVSL_OK) {
                const int s2 = S.status();
                if (s2 == EVSL_ERR_NOCONV) rc = ctx_fail(c, s2, "chebSI: some wanted pairs did not reach tol in %d passes",
                                                         o->maxit > 0 ? o->maxit : 100);
                else rc = status_message(c, s2, cap, 0);
            }
        }
    }
    cudaEventDestroy(ta);
    cudaEventDestroy(tb);
    return rc;
}

int drv_chebLanTr_batch(evsl_ctx *c, int njobs, evsl_slice_job *jobs, const evsl_lan_opts *o)
{
    evsl_batch *bt = nullptr;
    EVSL_TRY(batch_create(c, o, &bt));
    int rc = EVSL_OK;
    for (int j = 0; j < njobs && rc == EVSL_OK; j++) rc = batch_add(bt, &jobs[j]);
    int active = (int)bt->solvers.size();
    while (rc == EVSL_OK && active > 0) rc = batch_step(bt, &active, nullptr);
    batch_destroy(bt);
    if (rc != EVSL_OK) return rc;
    for (int j = 0; j < njobs; j++)
        if (jobs[j].status != EVSL_OK)
            return status_message(c, jobs[j].status, jobs[j].cap, o->maxit > 0 ? o->maxit : 20 * jobs[j].m);
    return EVSL_OK;
}
