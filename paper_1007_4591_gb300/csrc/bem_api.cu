// C-ABI entry points of libbem (declared in include/bem.h).
//
// Every entry point converts C++ exceptions into BEM_E* codes, records a
// message for bem_last_error(), and accepts host or device arrays: host
// arrays are staged through device buffers owned by the mesh.
#include <chrono>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <cstdlib>
#include <string>

#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "bem_internal.cuh"

namespace bem {

int gmres_solve(Mesh &m, const double *b, double *x, bool transpose, bem_solve_stats *st);
double energy_from_phi(Mesh &m, const double *phi_s);
void axpby(Mesh &m, double a, const double *x, double b, const double *y, double *out, int64_t n);
void adjoint_gradients(Mesh &m, double grad_out, double *dq_s, double *dx_s);

static thread_local std::string g_last_error = "no error";
void set_last_error(const std::string &msg) { g_last_error = msg; }

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of an input array (copied through `stage` when it lives on the host).
static const double *dev_in(Mesh &m, const double *p, size_t n, DArray<double> &stage) {
    if (is_device_ptr(p)) return p;
    if (stage.n < n) stage.alloc(n);
    BEM_CUDA(cudaMemcpyAsync(stage.p, p, n * sizeof(double), cudaMemcpyHostToDevice, m.stream));
    return stage.p;
}

struct OutArg {
    double *user;
    double *dev;
    size_t n;
    bool host;
};

static OutArg dev_out(Mesh &m, double *p, size_t n, DArray<double> &stage) {
    OutArg o{p, p, n, false};
    if (!is_device_ptr(p)) {
        if (stage.n < n) stage.alloc(n);
        o.dev = stage.p;
        o.host = true;
    }
    return o;
}

static void finish_out(Mesh &m, const OutArg &o) {
    if (o.host)
        BEM_CUDA(cudaMemcpyAsync(o.user, o.dev, o.n * sizeof(double), cudaMemcpyDeviceToHost, m.stream));
}

// Order the mesh's work stream after everything already queued on the
// caller's stream.
static void enter(Mesh &m) {
    BEM_CUDA(cudaEventRecord(m.ev_enter, m.user));
    BEM_CUDA(cudaStreamWaitEvent(m.stream, m.ev_enter, 0));
}

// Synchronise the mesh's stream and report a bounded device wait that ran
// out (the error word comes back in the same synchronisation).
static void sync(Mesh &m) {
    int *flag = reinterpret_cast<int *>(m.h_pinned + 7);  // the pinned buffer's last 8 bytes
    if (m.dev_err.p) BEM_CUDA(cudaMemcpyAsync(flag, m.dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, m.stream));
    BEM_CUDA(cudaStreamSynchronize(m.stream));
    if (m.dev_err.p && *flag) {
        *flag = 0;
        BEM_CUDA(cudaMemsetAsync(m.dev_err.p, 0, sizeof(int), m.stream));
        BEM_CUDA(cudaStreamSynchronize(m.stream));
        throw Error(BEM_ETIMEOUT, "a bounded device wait ran out (tensor-core M2L)");
    }
}

static std::atomic<size_t> g_dev_used{0}, g_dev_cap{0};

void dev_mem_reserve(size_t bytes) {
    const size_t cap = g_dev_cap.load();
    const size_t now = g_dev_used.fetch_add(bytes) + bytes;
    if (cap && now > cap) {
        g_dev_used.fetch_sub(bytes);
        throw Error(BEM_ENOMEM, "device memory cap of " + std::to_string(cap) + " bytes reached");
    }
}

void dev_mem_unreserve(size_t bytes) { g_dev_used.fetch_sub(bytes); }

// NVTX range around an entry point (shows up in Nsight timelines; a no-op
// without a tool attached)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

template <class F>
static int guarded(F &&f) {
    try {
        f();
        return BEM_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return BEM_ENOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return BEM_ECUDA;
    }
}

size_t Mesh::bytes() const {
    size_t b = tp.bytes() + tc.bytes();
    b += cen_perm.bytes() + cen64.bytes() + nrm64.bytes() + area64.bytes() + cen32.bytes() +
         nrm32.bytes() + cen64r.bytes() + nrm64r.bytes() + cen_key.bytes();
    b += qp_panel.bytes() + qpg64.bytes() + qw64.bytes() + qp32.bytes() + qp64r.bytes() + qp_key.bytes();
    b += chg_perm.bytes() + chgg64.bytes() + q64.bytes() + chg32.bytes() + chg64r.bytes() + chg_key.bytes();
    b += nt_off.bytes() + nt_col.bytes() + nt_val.bytes() + ntT_off.bytes() + ntT_col.bytes() +
         ntT_val.bytes() + qp_of_panel.bytes();
    if (tab) b += tab->bytes();
    if (tab2) b += tab2->bytes();
    b += Mf.bytes() + Lf.bytes() + Md.bytes() + Ld.bytes();
    b += lamq.bytes() + pan64.bytes() + cn_off.bytes() + cn_col.bytes() + cn_val.bytes() + cnT_off.bytes() + cnT_row.bytes() +
         cnT_val.bytes();
    b += Mtc.bytes() + ctq.bytes() + str32.bytes() + str64.bytes() + near64.bytes() + dpart_f.bytes() +
         dpart_d.bytes();
    b += xs.bytes() + ys.bytes() + zs.bytes() + far_f.bytes() + near_f.bytes() + far_d.bytes() +
         near_d.bytes() + io_a.bytes() + io_b.bytes() + red.bytes();
    b += dev_err.bytes();
    b += V.bytes() + H.bytes() + gv.bytes() + cs.bytes() + sn.bytes() + yv.bytes() + hv.bytes() +
         part.bytes() + sigma_s.bytes();
    return b;
}

template <class T>
static void ensure(DArray<T> &d, size_t n) {
    if (d.n < n) d.alloc(n);
}

// Work buffers (grow-only: a captured graph keeps pointing at them).
static void alloc_work(Mesh &m) {
    const size_t nc = (size_t)cell_stride(m.opt.p);
    const size_t ncell = (size_t)std::max(m.tp.ncell, m.tc.ncell);
    const size_t nt = (size_t)std::max<int64_t>(std::max<int64_t>(m.np, m.nc), m.nqp);
    if (m.opt.precision == BEM_MIXED) {
        ensure(m.Mf, ncell * nc);
        ensure(m.Lf, ncell * nc);
        ensure(m.far_f, nt);
        ensure(m.near_f, nt);
    } else {
        ensure(m.Md, ncell * nc);
        ensure(m.Ld, ncell * nc);
        ensure(m.far_d, nt);
        ensure(m.near_d, nt);
    }
    if (tc_m2l_available(m)) {
        ensure(m.Mtc, tc_staging_floats(m));
    }
    // near-field source pairs: each leaf padded to an even count
    const size_t nsrc = (size_t)std::max<int64_t>(m.nqp, m.nc) + (size_t)std::max(m.tp.nleaf, m.tc.nleaf) + 4;
    if (m.opt.precision == BEM_MIXED) ensure(m.str32, nsrc);
    else ensure(m.str64, nsrc);
    ensure(m.near64, (size_t)m.np);
    const size_t nv = (size_t)std::max<int64_t>(m.np, m.nc);
    ensure(m.xs, nv);
    ensure(m.ys, nv);
    ensure(m.zs, nv * 3);
    ensure(m.red, 16);
    if (!m.dev_err.p) {
        m.dev_err.alloc(2);  // [0] error word, [1] work-item counter of the tensor-core M2L
        BEM_CUDA(cudaMemsetAsync(m.dev_err.p, 0, 2 * sizeof(int), m.stream));
    }
    ensure(m.part, (size_t)(std::max(1, m.opt.gmres_restart) + 2) * 1024);
}

static void validate_options(const bem_options &o) {
    if (o.precision != BEM_MIXED && o.precision != BEM_FP64)
        throw Error(BEM_EINVAL, "precision must be BEM_MIXED or BEM_FP64");
    if (o.p < 1 || o.p > MAXP) throw Error(BEM_EINVAL, "expansion order p must be in 1..16");
    if (o.leaf_size < 1) throw Error(BEM_EINVAL, "leaf_size must be positive");
    if (o.depth > MORTON_BITS) throw Error(BEM_EINVAL, "depth must be <= 21");
    if (o.quad_points != 1 && o.quad_points != 7) throw Error(BEM_EINVAL, "quad_points must be 1 or 7");
    if (o.near_table < 0 || o.near_table > BEM_NEAR_EXACT) throw Error(BEM_EINVAL, "near_table must be 0, 1 or 2");
    if (o.galerkin != 0 && o.galerkin != 1) throw Error(BEM_EINVAL, "galerkin must be 0 or 1");
    if (o.gmres_restart < 1 || o.gmres_restart > 200) throw Error(BEM_EINVAL, "gmres_restart must be in 1..200");
    if (o.max_iter < 1) throw Error(BEM_EINVAL, "max_iter must be positive");
    if (!(o.tol > 0.0)) throw Error(BEM_EINVAL, "tol must be positive");
    if (o.charge_mode < 0 || o.charge_mode > 2) throw Error(BEM_EINVAL, "charge_mode must be 0, 1 or 2");
    if (o.m2l_mode < 0 || o.m2l_mode > 3) throw Error(BEM_EINVAL, "m2l_mode must be 0, 1, 2 or 3");
}

}  // namespace bem

using namespace bem;

struct bem_mesh : public bem::Mesh {};

extern "C" {

int bem_options_default(bem_options *opt) {
    if (!opt) {
        set_last_error("bem_options_default: NULL");
        return BEM_EINVAL;
    }
    opt->precision = BEM_MIXED;
    opt->p = 10;
    opt->leaf_size = 64;
    opt->depth = 0;
    opt->quad_points = 7;
    opt->gmres_restart = 30;
    opt->max_iter = 300;
    opt->tol = 1e-8;
    opt->flags = 0;
    opt->near_table = 1;
    opt->charge_mode = BEM_CHARGE_AUTO;
    opt->m2l_mode = BEM_M2L_AUTO;
    opt->graph = 0;
    opt->galerkin = 0;
    return BEM_OK;
}

int bem_mesh_create(const double *panels, int64_t n_p, const double *charges, int64_t n_c,
                    double eps_in, double eps_out, const bem_options *opt, void *stream,
                    bem_mesh **out) {
    Range rng("bem_mesh_create");
    if (!out) {
        set_last_error("bem_mesh_create: out is NULL");
        return BEM_EINVAL;
    }
    *out = nullptr;
    bem_mesh *m = nullptr;
    int rc = guarded([&] {
        if (!panels || n_p <= 0) throw Error(BEM_EINVAL, "need at least one panel");
        if (n_c < 0 || (n_c > 0 && !charges)) throw Error(BEM_EINVAL, "bad charge array");
        if (!(eps_in > 0.0) || !(eps_out > 0.0) || !std::isfinite(eps_in) || !std::isfinite(eps_out))
            throw Error(BEM_EINVAL, "permittivities must be positive and finite");
        if (n_p * 7 > (int64_t)INT32_MAX - 1024 || n_c > (int64_t)INT32_MAX - 1024)
            throw Error(BEM_EINVAL, "too many panels or charges for 32-bit indices");
        auto t0 = std::chrono::steady_clock::now();
        m = new bem_mesh();
        if (opt) m->opt = *opt;
        else bem_options_default(&m->opt);
        validate_options(m->opt);
        BEM_CUDA(cudaGetDevice(&m->device));
        m->user = (cudaStream_t)stream;
        // The far-field chain (small launches, each waiting on the last) runs at
        // the highest priority, the near field beside it at the lowest, so that
        // near-field blocks fill the SMs the chain leaves idle.
        int prio_lo = 0, prio_hi = 0;
        BEM_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        BEM_CUDA(cudaStreamCreateWithPriority(&m->stream, cudaStreamNonBlocking, prio_hi));
        BEM_CUDA(cudaStreamCreateWithPriority(&m->stream2, cudaStreamNonBlocking, prio_lo));
        BEM_CUDA(cudaEventCreateWithFlags(&m->ev_enter, cudaEventDisableTiming));
        BEM_CUDA(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
        BEM_CUDA(cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming));
        enter(*m);
        m->np = n_p;
        m->nc = n_c;
        m->nq = m->opt.quad_points;
        m->nqp = n_p * m->nq;
        m->eps_in = eps_in;
        m->eps_out = eps_out;
        m->ehat = 2.0 * (eps_in - eps_out) / (eps_in + eps_out);
        BEM_CUDA(cudaMallocHost((void **)&m->h_pinned, 64));
        DArray<double> sp, sc;
        // BEM_TIMING=1: the build steps' wall times on stderr (diagnostics)
        StepTimer st(m->stream);
        const double *dp = dev_in(*m, panels, (size_t)n_p * 9, sp);
        const double *dc = n_c > 0 ? dev_in(*m, charges, (size_t)n_c * 4, sc) : nullptr;
        st.mark("inputs to the device");
        build_geometry_and_trees(*m, dp, dc);
        keep_panel_vertices(*m, dp);
        st.mark("geometry, Morton sort, trees, lists");
        if (m->opt.galerkin) build_galerkin_geometry(*m);
        build_tables(*m);
        st.mark("translation tables");
        build_translation_groups(*m, m->tp);
        st.mark("panel tree: translation groups, near-field order");
        build_translation_groups(*m, m->tc);
        st.mark("charge tree: translation groups, near-field order");
        alloc_work(*m);
        st.mark("work buffers");
        if (m->opt.near_table) build_near_table(*m, dp);
        st.mark("near-singular table");
        build_charge_near(*m);
        build_ctq(*m);
        sync(*m);
        st.mark("C^T q");
        // last, so that its memory check sees everything else the mesh holds
        build_p2m_moments(*m, m->tp);
        st.mark("P2M panel moments");
        m->ms_build = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    });
    if (rc != BEM_OK) {
        if (m) {
            if (m->stream) cudaStreamSynchronize(m->stream);
            if (m->h_pinned) cudaFreeHost(m->h_pinned);
            if (m->stream2) cudaStreamSynchronize(m->stream2);
            cudaStream_t st = m->stream, st2 = m->stream2;
            cudaEvent_t ev = m->ev_enter, e1 = m->ev_fork, e2 = m->ev_join;
            delete m;
            for (cudaEvent_t e : {ev, e1, e2})
                if (e) cudaEventDestroy(e);
            if (st) cudaStreamDestroy(st);
            if (st2) cudaStreamDestroy(st2);
        }
        return rc;
    }
    *out = m;
    return BEM_OK;
}

int bem_mesh_destroy(bem_mesh *m) {
    if (!m) return BEM_OK;
    return guarded([&] {
        if (m->stream) cudaStreamSynchronize(m->stream);
        for (auto &e : m->tm.ev)
            if (e) cudaEventDestroy(e);
        for (auto &e : m->tm.kev)
            if (e) cudaEventDestroy(e);
        for (auto &e : m->tm.nev)
            if (e) cudaEventDestroy(e);
        if (m->h_pinned) cudaFreeHost(m->h_pinned);
        if (m->g_mv) cudaGraphExecDestroy(m->g_mv);
        if (m->stream2) cudaStreamSynchronize(m->stream2);
        cudaStream_t st = m->stream, st2 = m->stream2;
        cudaEvent_t ev = m->ev_enter, e1 = m->ev_fork, e2 = m->ev_join;
        delete m;
        for (cudaEvent_t e : {ev, e1, e2})
            if (e) cudaEventDestroy(e);
        if (st) cudaStreamDestroy(st);
        if (st2) cudaStreamDestroy(st2);
    });
}

int bem_set_charges(bem_mesh *m, const double *charges, int64_t n_c) {
    Range rng("bem_set_charges");
    if (!m) return BEM_EINVAL;
    return guarded([&] {
        enter(*m);
        if (n_c < 0 || (n_c > 0 && !charges)) throw Error(BEM_EINVAL, "bad charge array");
        DArray<double> sc;
        const double *dc = n_c > 0 ? dev_in(*m, charges, (size_t)n_c * 4, sc) : nullptr;
        m->nc = n_c;
        if (m->g_mv) {  // the charge tree's cells may change the shared buffers: recapture
            BEM_CUDA(cudaStreamSynchronize(m->stream));
            cudaGraphExecDestroy(m->g_mv);
            m->g_mv = nullptr;
        }
        rebuild_charge_tree(*m, dc);
        build_tables(*m);  // the charge tree's separation may have changed
        build_translation_groups(*m, m->tc);
        alloc_work(*m);
        build_charge_near(*m);
        build_ctq(*m);
        m->have_sigma = false;
        sync(*m);
    });
}

int bem_matvec(bem_mesh *m, const double *x, double *y) {
    Range rng("bem_matvec");
    if (!m || !x || !y) return BEM_EINVAL;
    return guarded([&] {
        enter(*m);
        const double *dx = dev_in(*m, x, m->np, m->io_a);
        gather_f64(dx, m->cen_perm.p, m->xs.p, m->np, m->stream);
        matvec_sorted(*m, m->xs.p, m->ys.p);
        OutArg o = dev_out(*m, y, m->np, m->io_b);
        scatter_f64(m->ys.p, m->cen_perm.p, o.dev, m->np, m->stream);
        finish_out(*m, o);
        sync(*m);
    });
}

int bem_matvec_t(bem_mesh *m, const double *x, double *y) {
    Range rng("bem_matvec_t");
    if (!m || !x || !y) return BEM_EINVAL;
    return guarded([&] {
        enter(*m);
        const double *dx = dev_in(*m, x, m->np, m->io_a);
        gather_f64(dx, m->cen_perm.p, m->xs.p, m->np, m->stream);
        matvec_t_sorted(*m, m->xs.p, m->ys.p);
        OutArg o = dev_out(*m, y, m->np, m->io_b);
        scatter_f64(m->ys.p, m->cen_perm.p, o.dev, m->np, m->stream);
        finish_out(*m, o);
        sync(*m);
    });
}

static void rhs_sorted(Mesh &m, double *b_s) {
    if (m.nc == 0) {
        BEM_CUDA(cudaMemsetAsync(b_s, 0, m.np * sizeof(double), m.stream));
        return;
    }
    charge_pass(m, SRC_CHARGE, m.opt.galerkin ? TGT_QUAD_DN : TGT_CEN_DN, nullptr, m.zs.p);
    axpby(m, -m.ehat, m.zs.p, 0.0, m.zs.p, b_s, m.np);
}

int bem_rhs(bem_mesh *m, double *b) {
    Range rng("bem_rhs");
    if (!m || !b) return BEM_EINVAL;
    return guarded([&] {
        enter(*m);
        rhs_sorted(*m, m->ys.p);
        OutArg o = dev_out(*m, b, m->np, m->io_b);
        scatter_f64(m->ys.p, m->cen_perm.p, o.dev, m->np, m->stream);
        finish_out(*m, o);
        sync(*m);
    });
}

int bem_solve(bem_mesh *m, const double *x0, double *sigma, bem_solve_stats *st) {
    Range rng("bem_solve");
    if (!m || !sigma) return BEM_EINVAL;
    int status = BEM_OK;
    int rc = guarded([&] {
        enter(*m);
        cudaEvent_t e0, e1, e2;
        BEM_CUDA(cudaEventCreate(&e0));
        BEM_CUDA(cudaEventCreate(&e1));
        BEM_CUDA(cudaEventCreate(&e2));
        BEM_CUDA(cudaEventRecord(e0, m->stream));
        if (m->sigma_s.n < (size_t)m->np) m->sigma_s.alloc(m->np);
        DArray<double> b;
        b.alloc(m->np);
        rhs_sorted(*m, b.p);
        BEM_CUDA(cudaEventRecord(e1, m->stream));
        if (x0) {
            const double *d0 = dev_in(*m, x0, m->np, m->io_a);
            gather_f64(d0, m->cen_perm.p, m->sigma_s.p, m->np, m->stream);
        } else {
            BEM_CUDA(cudaMemsetAsync(m->sigma_s.p, 0, m->np * sizeof(double), m->stream));
        }
        bem_solve_stats local{};
        status = gmres_solve(*m, b.p, m->sigma_s.p, false, &local);
        BEM_CUDA(cudaEventRecord(e2, m->stream));
        OutArg o = dev_out(*m, sigma, m->np, m->io_b);
        scatter_f64(m->sigma_s.p, m->cen_perm.p, o.dev, m->np, m->stream);
        finish_out(*m, o);
        sync(*m);
        float a = 0, c = 0;
        cudaEventElapsedTime(&a, e0, e1);
        cudaEventElapsedTime(&c, e1, e2);
        local.ms_rhs = a;
        local.ms_gmres = c;
        local.ms_total = a + c;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        m->have_sigma = true;
        if (st) *st = local;
        if (status != BEM_OK) set_last_error("GMRES did not reach the tolerance");
    });
    return rc != BEM_OK ? rc : status;
}

static double energy_sorted(Mesh &m, const double *sig_s, double *phi_user) {
    if (m.nc == 0) return 0.0;
    if (!phi_user && m.ctq_ok) return energy_from_ctq(m, sig_s);
    double *phi_s = m.zs.p;  // n_c <= 3 * max(n_p, n_c)
    charge_pass(m, SRC_QUAD, TGT_CHG_PHI, sig_s, phi_s);
    charge_near_phi(m, sig_s, phi_s, 1, 1);
    const double dG = energy_from_phi(m, phi_s);
    if (phi_user) {
        // phi_reac = (C sigma) / eps_in in the caller's charge order
        OutArg o = dev_out(m, phi_user, m.nc, m.io_b);
        axpby(m, 1.0 / m.eps_in, phi_s, 0.0, phi_s, m.ys.p, m.nc);
        scatter_f64(m.ys.p, m.chg_perm.p, o.dev, m.nc, m.stream);
        finish_out(m, o);
    }
    return dG;
}

int bem_energy(bem_mesh *m, const double *sigma, double *dG, double *phi) {
    Range rng("bem_energy");
    if (!m || !sigma) return BEM_EINVAL;
    return guarded([&] {
        enter(*m);
        const double *ds = dev_in(*m, sigma, m->np, m->io_a);
        gather_f64(ds, m->cen_perm.p, m->xs.p, m->np, m->stream);
        const double e = energy_sorted(*m, m->xs.p, phi);
        sync(*m);
        if (dG) *dG = e;
    });
}

int bem_bibee(bem_mesh *m, int variant, double *sigma_hat, double *dG) {
    Range rng("bem_bibee");
    if (!m) return BEM_EINVAL;
    return guarded([&] {
        enter(*m);
        double lam;
        if (variant == BEM_BIBEE_CFA) lam = -0.5;
        else if (variant == BEM_BIBEE_P) lam = 0.0;
        else if (variant == BEM_BIBEE_PLUS_HALF) lam = 0.5;
        else throw Error(BEM_EINVAL, "unknown BIBEE variant");
        // sigma_hat = -Ehat / (1 + Ehat lambda) (B q)
        const double f = -m->ehat / (1.0 + m->ehat * lam);
        if (m->nc == 0) BEM_CUDA(cudaMemsetAsync(m->xs.p, 0, m->np * sizeof(double), m->stream));
        else {
            charge_pass(*m, SRC_CHARGE, m->opt.galerkin ? TGT_QUAD_DN : TGT_CEN_DN, nullptr, m->zs.p);
            axpby(*m, f, m->zs.p, 0.0, m->zs.p, m->xs.p, m->np);
        }
        if (sigma_hat) {
            OutArg o = dev_out(*m, sigma_hat, m->np, m->io_b);
            scatter_f64(m->xs.p, m->cen_perm.p, o.dev, m->np, m->stream);
            finish_out(*m, o);
        }
        double e = energy_sorted(*m, m->xs.p, nullptr);
        sync(*m);
        if (dG) *dG = e;
    });
}

int bem_energy_backward(bem_mesh *m, double grad_out, double *dq, double *dx) {
    Range rng("bem_energy_backward");
    if (!m) return BEM_EINVAL;
    return guarded([&] {
        enter(*m);
        if (m->nc == 0) return;
        if (!m->have_sigma) {
            bem_solve_stats st{};
            if (m->sigma_s.n < (size_t)m->np) m->sigma_s.alloc(m->np);
            DArray<double> b;
            b.alloc(m->np);
            rhs_sorted(*m, b.p);
            BEM_CUDA(cudaMemsetAsync(m->sigma_s.p, 0, m->np * sizeof(double), m->stream));
            gmres_solve(*m, b.p, m->sigma_s.p, false, &st);
            m->have_sigma = true;
        }
        DArray<double> gq, gx;
        gq.alloc(m->nc);
        gx.alloc((size_t)m->nc * 3);
        adjoint_gradients(*m, grad_out, gq.p, gx.p);
        if (dq) {
            OutArg o = dev_out(*m, dq, m->nc, m->io_a);
            scatter_f64(gq.p, m->chg_perm.p, o.dev, m->nc, m->stream);
            finish_out(*m, o);
        }
        if (dx) {
            OutArg o = dev_out(*m, dx, (size_t)m->nc * 3, m->io_b);
            scatter_rows3(gx.p, m->chg_perm.p, o.dev, m->nc, m->stream);
            finish_out(*m, o);
        }
        sync(*m);
    });
}

int bem_mesh_info_get(const bem_mesh *m, bem_mesh_info *info) {
    if (!m || !info) return BEM_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->n_p = m->np;
    info->n_c = m->nc;
    info->depth = m->L;
    info->p = m->opt.p;
    info->precision = m->opt.precision;
    info->leaves = m->tp.nleaf;
    info->cells = m->tp.ncell;
    info->p2p_pairs = m->tp.p2p_pairs_cq;
    info->m2l_pairs = m->tp.nm2l;
    int64_t m2m = 0;
    if (m->tp.L >= 2) m2m = m->tp.ncell - m->tp.lvl_off[2];
    info->m2m_pairs = m2m;
    info->source_points = m->nqp;
    info->near_table_nnz = m->nt_nnz;
    info->root_side = m->side;
    info->device_bytes = m->bytes();
    info->ms_build = m->ms_build;
    info->p2m_segments = m->tp.p2m_seg_p >= 0 ? (int64_t)m->tp.p2m_seg_panel.n : 0;
    return BEM_OK;
}

int bem_set_wait_budget(bem_mesh *m, long long cycles) {
    if (!m || cycles < 0) return BEM_EINVAL;
    m->wait_budget = cycles > 0 ? cycles : 2000000000ll;
    return BEM_OK;
}

int bem_set_device_memory_cap(size_t bytes) {
    g_dev_cap.store(bytes);
    return BEM_OK;
}

int bem_set_profiling(bem_mesh *m, int enable) {
    if (!m) return BEM_EINVAL;
    return guarded([&] {
        if (enable && !m->tm.ev[0]) {
            for (auto &e : m->tm.ev) BEM_CUDA(cudaEventCreate(&e));
            for (auto &e : m->tm.kev) BEM_CUDA(cudaEventCreate(&e));
            for (auto &e : m->tm.nev) BEM_CUDA(cudaEventCreate(&e));
        }
        m->tm.on = enable != 0;
    });
}

int bem_last_phase_ms(const bem_mesh *m, double *times) {
    if (!m || !times) return BEM_EINVAL;
    if (!m->tm.on) {
        set_last_error("profiling is off");
        return BEM_EINVAL;
    }
    // phase k spans events beg[k] .. beg[k] + 1; with the near field run
    // before the fused L2P + epilogue, L2P is 5-6 and P2P 4-5
    int beg[7] = {0, 1, 2, 3, 4, 5, 6};
    if (m->tm.near_before_l2p) {
        beg[4] = 5;
        beg[5] = 4;
    }
    for (int k = 0; k < 7; ++k) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, m->tm.ev[beg[k]], m->tm.ev[beg[k] + 1]) != cudaSuccess) {
            cudaGetLastError();
            ms = 0;
        }
        times[k] = ms;
    }
    return BEM_OK;
}

int bem_last_m2l_ms(const bem_mesh *m, double *times) {
    if (!m || !times) return BEM_EINVAL;
    if (!m->tm.on || !m->tm.kev[0]) {
        set_last_error("profiling is off");
        return BEM_EINVAL;
    }
    for (int k = 0; k < 3; ++k) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, m->tm.kev[k], m->tm.kev[k + 1]) != cudaSuccess) {
            cudaGetLastError();  // not recorded (no tensor-core M2L in the last product)
            ms = 0;
        }
        times[k] = ms;
    }
    return BEM_OK;
}

int bem_last_near_ms(const bem_mesh *m, double *times) {
    if (!m || !times) return BEM_EINVAL;
    if (!m->tm.on || !m->tm.nev[0]) {
        set_last_error("profiling is off");
        return BEM_EINVAL;
    }
    for (int k = 0; k < 2; ++k) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, m->tm.nev[k], m->tm.nev[k + 1]) != cudaSuccess) {
            cudaGetLastError();  // not recorded (no near field in the last product)
            ms = 0;
        }
        times[k] = ms;
    }
    return BEM_OK;
}

const char *bem_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
