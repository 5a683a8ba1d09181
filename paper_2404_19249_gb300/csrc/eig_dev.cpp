// Device LOBPCG (Knyazev 2001) for the arrow-structured small pencil of
// Algorithm 3: the same iteration as the host solver (preconditioned
// residuals, W orthogonalised against X and B-normalised, exact
// recomputation of A and B times the new X and P, soft locking: converged
// wanted columns get no new search direction).  Two host round trips per
// iteration: the residual norms (convergence test, active columns) and the
// Rayleigh-Ritz step of the Gram matrices, which runs on the host (Cholesky,
// or the two-pass eigen-decomposition that drops near-dependent directions):
// GB300 executes 2 FP64 FMA per clock per SM, so a one-block FP64 dense
// eigensolver is about ten times slower than one host core (measured: 9.8 ms
// against ~0.9 ms for 78 columns).
#include "eig_dev.h"

#include <algorithm>
#include <cmath>
#include <utility>

#include "small_eig.h"

namespace nas {

int DevLobpcg::solve(const ArrowDev& A, const ArrowDev& B, const int32_t* diag_slot, int nev, int nguard,
                     double* lam, const double* U0, double* Uout, double tol, int maxit, cudaStream_t s,
                     const float* TH, bool reuse_block) {
    const int64_t m = A.nH + A.Na;
    if (nev < 1 || nev > m) return -1;
    const int k = (int)std::min<int64_t>(nev + nguard, m);
    const int kmax3 = 3 * k;
    if (m > m_cap || k > k_cap) {
        for (auto& b : bufs) b.alloc(m * k);
        T.alloc(m);
        theta.alloc(k);
        nrm.alloc(4 * k);
        int64_t gp = std::max<int64_t>({gram_tiles_partial_size(m, kmax3, 2 * kmax3),
                                        gram_tiles_partial_size(A.nH, 2 * std::max(1, A.Na), k),
                                        reduce_partial_size(3 * k)});
        gpart.alloc(gp);
        gtmp.alloc(2 * std::max(1, A.Na) * (int64_t)k);
        GAB.alloc((int64_t)kmax3 * 2 * kmax3);
        Y.alloc((int64_t)kmax3 * k);
        C.alloc((int64_t)k * k);
        Yp.alloc((int64_t)2 * k * k);
        actd.alloc(k);
        m_cap = m;
        k_cap = k;
    }
    if (TH) ppart.ensure(std::max<int64_t>(1, dense_precond_part_size(A.nH, k)));
    // pinned staging: [GA | GB] (kmax3 x 2 kmax3), norms (3k), Y (kmax3 k), Yp (2k k), theta (k), active (k ints)
    const size_t o_ga = 0, o_nrm = o_ga + 2 * (size_t)kmax3 * kmax3,
                 o_y = o_nrm + 3 * (size_t)k, o_yp = o_y + (size_t)kmax3 * k, o_th = o_yp + 2 * (size_t)k * k,
                 o_act = o_th + k, pin_need = o_act + k;
    if (pin_doubles < pin_need) {
        if (pin) cudaFreeHost(pin);
        pin = nullptr;
        NAS_CUDA(cudaMallocHost((void**)&pin, sizeof(double) * pin_need));
        pin_doubles = pin_need;
    }
    double* pGA = pin + o_ga;
    double* pN = pin + o_nrm;
    double* pY = pin + o_y;
    double* pYp = pin + o_yp;
    double* pTh = pin + o_th;
    int* pAct = reinterpret_cast<int*>(pin + o_act);
    double *X = bufs[0].p, *AX = bufs[1].p, *BX = bufs[2].p, *W = bufs[3].p, *AW = bufs[4].p, *BW = bufs[5].p;
    double *P = bufs[6].p, *AP = bufs[7].p, *BP = bufs[8].p, *X2 = bufs[9].p, *P2 = bufs[10].p;
    // A and B share the coarse pattern: both products in one pass over the input
    auto applyAB = [&](int w, const double* in, double* outA, double* outB) {
        launch_arrow_apply2(A, B, w, in, outA, outB, gpart.p, gtmp.p, s);
    };
    std::vector<double> hG, hH, hY, th, th_new, hn(3 * (size_t)k);
    // stream synchronisation, timed (host time spent waiting for the device)
    auto wait = [&]() {
        auto t0 = std::chrono::steady_clock::now();
        NAS_CUDA(cudaStreamSynchronize(s));
        wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    // Rayleigh-Ritz on the basis S (ns columns): Grams on the device, the rest on the host
    // both Grams in one pass: S^T [AS | BS] -> [ns][2 ns], split into GA and GB
    auto grams = [&](const ColBlocks& S, const ColBlocks& AS, const ColBlocks& BS) {
        ColBlocks R = AS;
        for (int u = 0; u < BS.nblk; ++u) R.add(BS.p[u], BS.ld[u], BS.w[u]);
        launch_gram_tiles(m, S, R, gpart.p, GAB.p, s);
    };
    auto fetch = [&](int ns, bool norms) {
        NAS_CUDA(cudaMemcpyAsync(pGA, GAB.p, sizeof(double) * ns * 2 * ns, cudaMemcpyDeviceToHost, s));
        if (norms) NAS_CUDA(cudaMemcpyAsync(pN, nrm.p, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost, s));
        wait();
        hH.resize((size_t)ns * ns);
        hG.resize((size_t)ns * ns);
        for (int a = 0; a < ns; ++a) {
            std::copy(pGA + (size_t)a * 2 * ns, pGA + (size_t)a * 2 * ns + ns, hH.begin() + (size_t)a * ns);
            std::copy(pGA + (size_t)a * 2 * ns + ns, pGA + (size_t)(a + 1) * 2 * ns, hG.begin() + (size_t)a * ns);
        }
        if (norms) hn.assign(pN, pN + 3 * (size_t)k);
    };
    // host Rayleigh-Ritz from the fetched Grams (fallback and large ns)
    auto rr_host = [&](int ns, std::vector<double>& th_out) {
        auto t0 = std::chrono::steady_clock::now();
        bool fb = false;
        int r = rayleigh_ritz_grams(ns, hG, hH, k, hY, th_out, &fb);
        ++rr_calls;
        if (fb) ++rr_fallbacks;
        rr_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (r == 0) {
            // from the pinned area: it is rewritten only after the next synchronisation
            std::copy(hY.begin(), hY.begin() + (size_t)ns * k, pY);
            std::copy(th_out.begin(), th_out.begin() + k, pTh);
            NAS_CUDA(cudaMemcpyAsync(Y.p, pY, sizeof(double) * ns * k, cudaMemcpyHostToDevice, s));
            NAS_CUDA(cudaMemcpyAsync(theta.p, pTh, sizeof(double) * k, cudaMemcpyHostToDevice, s));
        }
        return r;
    };
    // Rayleigh-Ritz of the basis whose Grams are in GA/GB, on the host; with
    // norms = true the residual norms of the current X come with the same
    // round trip.  th_out receives the new Ritz values; Y/theta on the device
    // hold the result.
    auto rr = [&](int ns, bool norms, std::vector<double>& th_out) {
        th_out.resize(k);
        fetch(ns, norms);
        return rr_host(ns, th_out);
    };
    // ---- start.  reuse_block: the whole block of the previous solve (same m,
    // k and F_B; its columns are B-orthonormal Ritz vectors of a nearby F_A),
    // with Rayleigh quotients as the first Ritz values - no start-up
    // Rayleigh-Ritz.  Otherwise warm vectors for the wanted columns and
    // deterministic pseudo-random ones (generated once per (m, k)) for the rest,
    // B-orthonormalised by a Rayleigh-Ritz step.
    const bool reuse = reuse_block && keep_m == m && keep_k == k;
    if (reuse) {
        NAS_CUDA(cudaMemcpyAsync(X, Xkeep.p, sizeof(double) * m * k, cudaMemcpyDeviceToDevice, s));
        applyAB(k, X, AX, BX);
        const double* Xs[2] = {X, X};
        const double* Ys[2] = {AX, BX};
        launch_coldots(m, k, 2, Xs, Ys, nullptr, gpart.p, nrm.p, s);
        NAS_CUDA(cudaMemcpyAsync(pN, nrm.p, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, s));
        wait();
        th.resize(k);
        for (int j = 0; j < k; ++j) th[j] = pN[j] / (pN[k + j] > 0.0 ? pN[k + j] : 1.0);
        std::copy(th.begin(), th.end(), pTh);
        NAS_CUDA(cudaMemcpyAsync(theta.p, pTh, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    } else {
        if (x0_m != m || x0_k != k) {
            std::vector<double> h((size_t)m * k);
            for (int64_t i = 0; i < m; ++i)
                for (int j = 0; j < k; ++j) {
                    double r = std::sin(12.9898 * (i + 1) + 78.233 * (j + 1)) * 43758.5453;
                    h[i * k + j] = r - std::floor(r) - 0.5;
                }
            X0.alloc(m * k);
            NAS_CUDA(cudaMemcpyAsync(X0.p, h.data(), sizeof(double) * m * k, cudaMemcpyHostToDevice, s));
            NAS_CUDA(cudaStreamSynchronize(s));  // the host copy must outlive the upload
            x0_m = m;
            x0_k = k;
        }
        NAS_CUDA(cudaMemcpyAsync(X, X0.p, sizeof(double) * m * k, cudaMemcpyDeviceToDevice, s));
        if (U0)
            NAS_CUDA(cudaMemcpy2DAsync(X, sizeof(double) * k, U0, sizeof(double) * nev, sizeof(double) * nev, m,
                                       cudaMemcpyDeviceToDevice, s));
        applyAB(k, X, AX, BX);
        ColBlocks S = ColBlocks::one(X, k, k), AS = ColBlocks::one(AX, k, k), BS = ColBlocks::one(BX, k, k);
        grams(S, AS, BS);
        if (rr(k, false, th) != 0) return -1;
        launch_cols_mult(m, S, Y.p, k, 1.0, 0.0, X2, s);
        std::swap(X, X2);
        applyAB(k, X, AX, BX);
    }
    {
        const double sigma = th[0] - 0.1 * std::fabs(th[0]) - 1.0;
        launch_eig_precond(A, B, diag_slot, sigma, T.p, s);
    }
    int np = 0;
    int it = 0;
    std::vector<int> act;
    std::vector<double> hYp;
    for (; it < maxit; ++it) {
        // residual R = AX - BX theta of the current X (into X2, free until the
        // update below) and its norms: one round trip decides convergence and
        // the active columns (soft locking: unconverged wanted columns and
        // every guard column get a new search direction)
        double* R = X2;
        launch_eig_resid(m, k, AX, BX, theta.p, R, s);
        {
            const double* Xs[3] = {R, AX, BX};
            launch_coldots(m, k, 3, Xs, Xs, nullptr, gpart.p, nrm.p, s);
        }
        NAS_CUDA(cudaMemcpyAsync(pN, nrm.p, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost, s));
        wait();
        hn.assign(pN, pN + 3 * (size_t)k);
        double worst = 0.0;
        std::vector<double> rel(k);
        for (int j = 0; j < k; ++j) {
            rel[j] = std::sqrt(std::max(hn[j], 0.0)) /
                     (std::sqrt(std::max(hn[k + j], 0.0)) +
                      std::fabs(th[j]) * std::sqrt(std::max(hn[2 * k + j], 0.0)) + 1e-300);
            if (j < nev) worst = std::max(worst, rel[j]);
        }
        if (!std::isfinite(worst)) return -1;
        if (worst <= tol) break;
        act.clear();
        for (int j = 0; j < k; ++j)
            if (j >= nev || rel[j] > 0.1 * tol) act.push_back(j);
        const int ka = (int)act.size();
        std::copy(act.begin(), act.end(), pAct);
        NAS_CUDA(cudaMemcpyAsync(actd.p, pAct, sizeof(int) * ka, cudaMemcpyHostToDevice, s));
        // W = T R(:, act)
        launch_gather_cols(m, k, ka, actd.p, R, P2, s);
        if (TH)
            (tc ? launch_dense_precond_tc : launch_dense_precond)(A.nH, m, ka, TH, P2, T.p, ppart.p, W, s);
        else
            launch_scale_rows(m, ka, T.p, P2, W, s);
        // W <- W - X (BX^T W), then unit B-norm columns (AW scaled alike)
        launch_gram_tiles(m, ColBlocks::one(BX, k, k), ColBlocks::one(W, ka, ka), gpart.p, C.p, s);
        launch_cols_mult(m, ColBlocks::one(X, k, k), C.p, ka, -1.0, 1.0, W, s);
        applyAB(ka, W, AW, BW);
        {
            const double* Xs[1] = {W};
            const double* Ys[1] = {BW};
            launch_coldots(m, ka, 1, Xs, Ys, nullptr, gpart.p, nrm.p + 3 * k, s);
        }
        launch_inv_sqrt_scale(m, ka, nrm.p + 3 * k, W, BW, AW, s);
        ColBlocks S = ColBlocks::one(X, k, k), AS = ColBlocks::one(AX, k, k), BS = ColBlocks::one(BX, k, k);
        S.add(W, ka, ka);
        AS.add(AW, ka, ka);
        BS.add(BW, ka, ka);
        if (np > 0) {
            S.add(P, np, np);
            AS.add(AP, np, np);
            BS.add(BP, np, np);
        }
        const int ns = S.ncols();
        grams(S, AS, BS);
        if (rr(ns, false, th_new) != 0) {
            if (np == 0) return -1;
            np = 0;  // restart without P
            continue;
        }
        th.swap(th_new);
        // new X = S Y; new P = [W, P] part of S Y for the active columns
        launch_cols_mult(m, S, Y.p, k, 1.0, 0.0, X2, s);
        {
            const int nwp = ns - k;
            hYp.assign((size_t)nwp * ka, 0.0);
            for (int a = 0; a < nwp; ++a)
                for (int q = 0; q < ka; ++q) hYp[(size_t)a * ka + q] = hY[(size_t)(k + a) * k + act[q]];
            std::copy(hYp.begin(), hYp.end(), pYp);
            NAS_CUDA(cudaMemcpyAsync(Yp.p, pYp, sizeof(double) * nwp * ka, cudaMemcpyHostToDevice, s));
            ColBlocks WP = ColBlocks::one(W, ka, ka);
            if (np > 0) WP.add(P, np, np);
            launch_cols_mult(m, WP, Yp.p, ka, 1.0, 0.0, P2, s);
        }
        std::swap(X, X2);
        std::swap(P, P2);
        np = ka;
        // exact images (implicitly updated ones drift and break the Rayleigh-Ritz)
        applyAB(k, X, AX, BX);
        applyAB(np, P, AP, BP);
        {
            const double* Xs[1] = {P};
            const double* Ys[1] = {BP};
            launch_coldots(m, np, 1, Xs, Ys, nullptr, gpart.p, nrm.p + 3 * k, s);
        }
        launch_inv_sqrt_scale(m, np, nrm.p + 3 * k, P, AP, BP, s);
    }
    if (it >= maxit) return -1;
    // X holds B-orthonormal Ritz vectors (every iteration ends with X = S Y):
    // the wanted columns are the output; the whole block is kept for the next
    // solve of the same pencil family
    NAS_CUDA(cudaMemcpy2DAsync(Uout, sizeof(double) * nev, X, sizeof(double) * k, sizeof(double) * nev, m,
                               cudaMemcpyDeviceToDevice, s));
    Xkeep.ensure((size_t)m * k);
    NAS_CUDA(cudaMemcpyAsync(Xkeep.p, X, sizeof(double) * m * k, cudaMemcpyDeviceToDevice, s));
    keep_m = m;
    keep_k = k;
    for (int j = 0; j < nev; ++j) lam[j] = th[j];
    return it;
}

}  // namespace nas
