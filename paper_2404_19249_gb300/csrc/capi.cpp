// C ABI of the nas library (include/nas.h): argument checks, exception to
// status-code translation, and the context lifecycle.
#include <omp.h>

#include <atomic>
#include <cstring>
#include <new>
#include <set>
#include <thread>

#include "ctx.h"

using nas::Error;

namespace {

template <class F>
int guarded(nas_ctx* c, F&& f) {
    if (!c) return NAS_E_INVALID_ARG;
    try {
        int r = f();
        if (r == NAS_OK) c->err.clear();
        return r;
    } catch (const Error& e) {
        c->err = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        c->err = "host allocation failed";
        return NAS_E_OOM;
    } catch (const std::exception& e) {
        c->err = e.what();
        return NAS_E_CUDA;
    }
}

void invalidate(nas_ctx* c) {
    ++c->state_id;
    c->setup_done = false;
    c->initialized = false;
    c->anl_valid = false;
}

template <typename T>
int spmm_layout_call(int layout, int64_t n_rows, const int32_t* row_ptr, const int32_t* col, const T* val,
                            int N, const T* X, T* Y, void* stream) {
    if (n_rows < 0 || N < 1 || !row_ptr || !col || !val || !X || !Y) return NAS_E_INVALID_ARG;
    try {
        nas::launch_spmm_layout(layout, n_rows, row_ptr, col, val, N, X, Y, static_cast<cudaStream_t>(stream));
        return NAS_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

}  // namespace

extern "C" {

void nas_default_options(nas_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mu = -1.0;
    o->tol_bvp = 1e-12;
    o->tol_poisson = 1e-12;
    o->tol_scf = 1e-8;
    o->tol_inner = 1e-8;
    o->max_cg = 2000;
    o->max_poisson = 20000;
    o->max_inner = 50;
    o->max_outer = 100;
    o->anderson_depth = 5;
    o->anderson_beta = 0.7;
    o->hartree = 1;
    o->xc = 1;
    o->multipole = 0;
    o->omega = 1.0;
    o->check_every = 1;
    o->timing = 0;
    o->eig_dense_max = 1200;
    o->eig_tol = -1.0;
    o->spmv_lanes = 0;
    o->eig_device = 1;
    o->eig_precond = 1;
    o->eig_adapt = 1e-3;
    o->poisson_sell = 1;
    o->poisson_adaptive = 0;
    o->poisson_fused = 0;
    o->poisson_two_level = 1;
    o->precision = 0;
    o->smearing = 0.0;
    o->inner_adapt = 0.0;
    o->bvp_two_level = 0;
    o->bvp_adapt = 0.0;
    o->anderson_restart = 0.0;
    o->poisson_f32 = 0;
    o->dense_tc = 1;
    o->density_pairs = 0;
}

const char* nas_version(void) { return "nas 0.1 (sm_103a, FP64)"; }

int nas_create(nas_ctx** out, int device, void* cuda_stream) {
    if (!out) return NAS_E_INVALID_ARG;
    *out = nullptr;
    nas_ctx* c = new (std::nothrow) nas_ctx();
    if (!c) return NAS_E_OOM;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        delete c;
        return NAS_E_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return NAS_E_CUDA;
    }
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    nas_default_options(&c->opt);
    *out = c;
    return NAS_OK;
}

void nas_destroy(nas_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& p : c->ev_pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->pcg1_exec) cudaGraphExecDestroy(c->pcg1_exec);
    if (c->pcg1f_exec) cudaGraphExecDestroy(c->pcg1f_exec);
    for (auto e : c->pcg1_ev) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

const char* nas_last_error(const nas_ctx* c) { return c ? c->err.c_str() : "null context"; }

int nas_set_mesh(nas_ctx* c, int which, int order, int64_t n_vert, const double* xyz, int64_t n_tet,
                 const int32_t* tet) {
    return guarded(c, [&]() {
        if (!xyz || !tet || n_vert < 4 || n_tet < 1) nas::fail(NAS_E_INVALID_ARG, "empty mesh");
        if (which == NAS_FINE) {
            if (order != 1 && order != 2) nas::fail(NAS_E_INVALID_ARG, "fine order must be 1 or 2");
            c->fxyz.assign(xyz, xyz + 3 * n_vert);
            c->ftet.assign(tet, tet + 4 * n_tet);
            c->fnv = n_vert;
            c->fne = n_tet;
            c->fine_order = order;
            c->have_fine = true;
        } else if (which == NAS_COARSE) {
            if (order != 1) nas::fail(NAS_E_INVALID_ARG, "coarse space is P1");
            c->cxyz.assign(xyz, xyz + 3 * n_vert);
            c->ctet.assign(tet, tet + 4 * n_tet);
            c->cnv = n_vert;
            c->cne = n_tet;
            c->have_coarse = true;
        } else {
            nas::fail(NAS_E_INVALID_ARG, "which must be NAS_FINE or NAS_COARSE");
        }
        for (int64_t i = 0; i < 4 * n_tet; ++i)
            if (tet[i] < 0 || tet[i] >= n_vert) nas::fail(NAS_E_MESH, "vertex id out of range");
        invalidate(c);
        return NAS_OK;
    });
}

int nas_set_system(nas_ctx* c, int n_nuc, const double* R, const double* Z, int potential, double smooth_a,
                   int n_orb, const double* occ) {
    return guarded(c, [&]() {
        if (n_nuc < 0 || (n_nuc > 0 && (!R || !Z))) nas::fail(NAS_E_INVALID_ARG, "nuclei");
        if (n_orb < 1 || n_orb > 64) nas::fail(NAS_E_INVALID_ARG, "n_orb must be in 1..64");
        if (potential < NAS_POT_COULOMB || potential > NAS_POT_HARMONIC) nas::fail(NAS_E_INVALID_ARG, "potential");
        if (potential == NAS_POT_SMOOTHED && !(smooth_a > 0.0)) nas::fail(NAS_E_INVALID_ARG, "smooth_a must be > 0");
        std::vector<double> occv(occ ? occ : (const double*)nullptr, occ ? occ + n_orb : (const double*)nullptr);
        if (!occ) occv.assign(n_orb, 2.0);
        if (c->setup_done && n_nuc == c->n_nuc && n_orb == c->N && potential == c->potential &&
            smooth_a == c->smooth_a && occv == c->occ) {
            // only the nuclei move or change charge: keep the mesh structures
            c->R.assign(R, R + 3 * n_nuc);
            c->Z.assign(Z, Z + n_nuc);
            ++c->state_id;
            nas::ctx_update_nuclei(c);
            return NAS_OK;
        }
        c->n_nuc = n_nuc;
        c->R.assign(R ? R : (const double*)nullptr, R ? R + 3 * n_nuc : (const double*)nullptr);
        c->Z.assign(Z ? Z : (const double*)nullptr, Z ? Z + n_nuc : (const double*)nullptr);
        c->potential = potential;
        c->smooth_a = smooth_a;
        c->N = n_orb;
        if (occ)
            c->occ.assign(occ, occ + n_orb);
        else
            c->occ.assign(n_orb, 2.0);
        c->lam.assign(n_orb, 0.0);
        c->have_system = true;
        invalidate(c);
        return NAS_OK;
    });
}

int nas_set_options(nas_ctx* c, const nas_options* o) {
    return guarded(c, [&]() {
        if (!o) nas::fail(NAS_E_INVALID_ARG, "null options");
        if (o->tol_bvp <= 0 || o->tol_poisson <= 0 || o->max_cg < 1 || o->max_poisson < 1 || o->max_inner < 1 ||
            o->anderson_depth < 1 || o->anderson_depth > 16 || o->precision < 0 || o->precision > 1 ||
            o->eig_device < 0 || o->eig_device > 1 || o->poisson_adaptive < 0 || o->poisson_adaptive > 1 ||
            !(o->eig_adapt > 0.0) || o->eig_adapt > 1.0 || o->eig_precond < 0 || o->eig_precond > 2 ||
            o->poisson_sell < 0 || o->poisson_sell > 1 || o->poisson_fused < 0 || o->poisson_fused > 1 ||
            !(o->smearing >= 0.0) || !(o->inner_adapt >= 0.0) || o->bvp_two_level < 0 || o->bvp_two_level > 1 ||
            !(o->bvp_adapt >= 0.0) || !(o->anderson_restart >= 0.0) ||
            o->poisson_f32 < 0 || o->poisson_f32 > 1 || o->dense_tc < 0 || o->dense_tc > 1 ||
            o->density_pairs < 0 || o->density_pairs > 1)
            nas::fail(NAS_E_INVALID_ARG, "options out of range");
        bool rebuild = (o->mu != c->opt.mu) || (o->omega != c->opt.omega) ||
                       (o->poisson_two_level != c->opt.poisson_two_level) || (o->eig_precond != c->opt.eig_precond);
        c->opt = *o;
        ++c->state_id;
        if (rebuild && c->setup_done) invalidate(c);
        return NAS_OK;
    });
}

int nas_init(nas_ctx* c, const double* psi0) {
    return guarded(c, [&]() {
        NAS_CUDA(cudaSetDevice(c->device));
        ++c->state_id;
        if (!c->setup_done) nas::ctx_setup(c);
        nas::ctx_init(c, psi0);
        return NAS_OK;
    });
}

int nas_step(nas_ctx* c, nas_report* rep) {
    return guarded(c, [&]() {
        NAS_CUDA(cudaSetDevice(c->device));
        ++c->state_id;
        return nas::ctx_step(c, rep);
    });
}

int nas_solve(nas_ctx* c, nas_report* rep) {
    return guarded(c, [&]() {
        NAS_CUDA(cudaSetDevice(c->device));
        ++c->state_id;
        int status = NAS_OK;
        nas_report r{};
        bool done = false;
        for (int l = 0; l < c->opt.max_outer && !done; ++l) {
            status = nas::ctx_step(c, &r);
            done = r.drho < c->opt.tol_scf;
        }
        if (rep) *rep = r;
        return (status == NAS_OK && !done) ? NAS_E_NOT_CONVERGED : status;
    });
}

int nas_batch_run(nas_ctx** ctxs, int count, int steps, int n_threads, int* status, nas_report* reports) {
    if (count < 0 || n_threads < 1 || (count > 0 && (!ctxs || !status))) return NAS_E_INVALID_ARG;
    if (count == 0) return NAS_OK;
    std::set<nas_ctx*> seen;
    for (int i = 0; i < count; ++i) {
        nas_ctx* c = ctxs[i];
        if (!c || !seen.insert(c).second) {
            if (ctxs[0]) ctxs[0]->err = "nas_batch_run: null or repeated context";
            return NAS_E_INVALID_ARG;
        }
        if (!c->initialized || c->device != ctxs[0]->device) {
            ctxs[0]->err = c->err = "nas_batch_run: contexts must be initialised and on one device";
            return NAS_E_INVALID_ARG;
        }
    }
    // Each context runs on a private non-blocking stream for the duration of
    // the batch, ordered after the work already queued on its own stream, and
    // its own stream waits for the batch's work at the end.
    if (cudaSetDevice(ctxs[0]->device) != cudaSuccess) return NAS_E_CUDA;
    std::vector<cudaStream_t> own(count), priv(count, nullptr);
    for (int i = 0; i < count; ++i) {
        nas_ctx* c = ctxs[i];
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&priv[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(e, c->stream) != cudaSuccess ||
            cudaStreamWaitEvent(priv[i], e, 0) != cudaSuccess) {
            for (int j = 0; j <= i; ++j)
                if (priv[j]) cudaStreamDestroy(priv[j]);
            if (e) cudaEventDestroy(e);
            return NAS_E_CUDA;
        }
        cudaEventDestroy(e);
        own[i] = c->stream;
        c->stream = priv[i];
        c->concurrent = true;  // solves run at the same time: no cooperative launches
    }
    const int nt = std::min(n_threads, count);
    const int omp_each = std::max(1, omp_get_max_threads() / nt);
    std::atomic<int> next{0};
    auto worker = [&]() {
        omp_set_num_threads(omp_each);
        for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
            nas_report r{};
            int st = NAS_OK;
            if (steps > 0) {
                for (int k = 0; k < steps; ++k) {
                    st = nas_step(ctxs[i], &r);
                    if (st < 0 && st != NAS_E_NOT_CONVERGED) break;
                }
            } else {
                st = nas_solve(ctxs[i], &r);
            }
            status[i] = st;
            if (reports) reports[i] = r;
        }
    };
    // workers are new threads, so the caller's OpenMP settings stay as they were
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    int rc = NAS_OK;
    for (int i = 0; i < count; ++i) {
        nas_ctx* c = ctxs[i];
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(e, priv[i]) != cudaSuccess ||
            cudaStreamWaitEvent(own[i], e, 0) != cudaSuccess)
            rc = NAS_E_CUDA;
        if (e) cudaEventDestroy(e);
        c->stream = own[i];
        c->concurrent = false;
        cudaStreamDestroy(priv[i]);  // released once its queued work completes
    }
    return rc;
}

int nas_get(nas_ctx* c, int what, void* dst, size_t bytes, int on_device) {
    return guarded(c, [&]() {
        if (!dst) nas::fail(NAS_E_INVALID_ARG, "null destination");
        NAS_CUDA(cudaSetDevice(c->device));
        nas::ctx_get(c, what, dst, bytes, on_device);
        return NAS_OK;
    });
}

int nas_set_state(nas_ctx* c, const double* lam, const double* psi, const double* rho_in, int on_device) {
    return guarded(c, [&]() {
        NAS_CUDA(cudaSetDevice(c->device));
        ++c->state_id;
        nas::ctx_set_state(c, lam, psi, rho_in, on_device);
        return NAS_OK;
    });
}

int nas_apply(nas_ctx* c, int op, const void* in, int64_t cnt, void* out, int on_device) {
    return guarded(c, [&]() {
        NAS_CUDA(cudaSetDevice(c->device));
        nas::ctx_apply(c, op, in, cnt, out, on_device);
        return NAS_OK;
    });
}

int nas_spmm_f64(int64_t n_rows, const int32_t* row_ptr, const int32_t* col, const double* val, int N,
                 const double* X, double* Y, void* stream) {
    if (n_rows < 0 || N < 1 || !row_ptr || !col || !val || !X || !Y) return NAS_E_INVALID_ARG;
    try {
        nas::Csr A{n_rows, row_ptr, col, val};
        nas::launch_spmm(A, N, X, Y, 1.0, 0.0, static_cast<cudaStream_t>(stream));
        return NAS_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

int nas_reconstruct_f64(int tc, int64_t n, const int32_t* icol, const double* ival, int N, const double* U,
                        int64_t nH, int Na, const double* Uhat, double* Psi, void* stream) {
    if (n < 0 || N < 1 || Na < 1 || nH < 0 || !icol || !ival || !U || !Uhat || !Psi) return NAS_E_INVALID_ARG;
    if (tc && !nas::reconstruct_tc_supported(N, Na)) return NAS_E_INVALID_ARG;
    if (n == 0) return NAS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    try {
        if (tc) {
            nas::launch_reconstruct_tc(n, icol, ival, N, U, nH, Na, Uhat, Psi, s);
            if (nas::tc_error_take(s)) return NAS_E_CUDA;
        } else {
            nas::launch_reconstruct(n, icol, ival, N, U, nH, Na, Uhat, Psi, s);
        }
    } catch (const Error& e) {
        return e.code;
    }
    return NAS_OK;
}

int nas_gram_sym_f64(int tc, int64_t n, int N, const double* X, const double* Y, double* G, void* stream) {
    if (n < 0 || N < 1 || (int64_t)N * (N + 1) / 2 > 16 * 256 || !X || !Y || !G) return NAS_E_INVALID_ARG;
    if (tc && !nas::gram_tc_supported(N)) return NAS_E_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* part = nullptr;
    const size_t bytes = sizeof(double) * (size_t)nas::reduce_partial_size((int64_t)N * N);
    if (cudaMallocAsync(reinterpret_cast<void**>(&part), bytes, s) != cudaSuccess) return NAS_E_CUDA;
    int rc = NAS_OK;
    try {
        if (tc) {
            nas::launch_gram_sym_tc(n, N, X, Y, part, G, s);
            if (nas::tc_error_take(s)) rc = NAS_E_CUDA;
        } else {
            nas::launch_gram_sym(n, N, X, Y, part, G, s);
        }
    } catch (const Error& e) {
        rc = e.code;
    }
    if (cudaFreeAsync(part, s) != cudaSuccess && rc == NAS_OK) rc = NAS_E_CUDA;
    return rc;
}

int nas_dense_precond_f32(int tc, int64_t nH, int k, const float* T, const double* R, double* W, void* stream) {
    if (nH < 0 || k < 1 || k > 256 || !T || !R || !W) return NAS_E_INVALID_ARG;
    if (nH == 0) return NAS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* part = nullptr;
    const size_t bytes = sizeof(float) * (size_t)nas::dense_precond_part_size(nH, k);
    if (cudaMallocAsync(reinterpret_cast<void**>(&part), bytes, s) != cudaSuccess) return NAS_E_CUDA;
    int rc = NAS_OK;
    try {
        if (tc) {
            nas::launch_dense_precond_tc(nH, nH, k, T, R, nullptr, part, W, s);
            if (nas::tc_error_take(s)) rc = NAS_E_CUDA;
        } else {
            nas::launch_dense_precond(nH, nH, k, T, R, nullptr, part, W, s);
        }
    } catch (const Error& e) {
        rc = e.code;
    }
    if (cudaFreeAsync(part, s) != cudaSuccess && rc == NAS_OK) rc = NAS_E_CUDA;
    return rc;
}

int nas_spmm_layouts(void) { return nas::spmm_num_layouts(); }

const char* nas_spmm_layout_name(int layout) { return nas::spmm_layout_name(layout); }

int nas_spmm_tuning(char* buf, size_t bytes) {
    const std::string r = nas::spmm_tuning_report();
    if (buf && bytes > 0) {
        const size_t k = std::min(bytes - 1, r.size());
        std::memcpy(buf, r.data(), k);
        buf[k] = '\0';
    }
    return (int)r.size();
}

int nas_spmm_f64_layout(int layout, int64_t n_rows, const int32_t* row_ptr, const int32_t* col, const double* val,
                        int N, const double* X, double* Y, void* stream) {
    return spmm_layout_call(layout, n_rows, row_ptr, col, val, N, X, Y, stream);
}

int nas_spmm_f32_layout(int layout, int64_t n_rows, const int32_t* row_ptr, const int32_t* col, const float* val,
                        int N, const float* X, float* Y, void* stream) {
    return spmm_layout_call(layout, n_rows, row_ptr, col, val, N, X, Y, stream);
}

int nas_coldot_f64(int64_t n, int N, const double* X, const double* Y, const double* w, double* out,
                   void* stream) {
    if (n < 0 || N < 1 || N > 256 || !X || !Y || !out) return NAS_E_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* partial = nullptr;
    size_t bytes = sizeof(double) * (size_t)nas::reduce_partial_size(N);
    if (cudaMallocAsync(reinterpret_cast<void**>(&partial), bytes, s) != cudaSuccess) return NAS_E_CUDA;
    int rc = NAS_OK;
    try {
        const double* Xs[1] = {X};
        const double* Ys[1] = {Y};
        nas::launch_coldots(n, N, 1, Xs, Ys, w, partial, out, s);
    } catch (const Error& e) {
        rc = e.code;
    }
    if (cudaFreeAsync(partial, s) != cudaSuccess && rc == NAS_OK) rc = NAS_E_CUDA;
    return rc;
}

}  // extern "C"
