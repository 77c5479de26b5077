// C ABI of the hyperbolic self-gravity library (declarations and contracts in include/hg.h).
// Host-side runtime: argument checks, device buffers, the sub-step loop and state movement.  Every arithmetic
// step of the method runs in the kernels of stencil.cu, temporal.cu, boundary.cu and fields.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "hg_internal.cuh"

namespace hg {

static thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(HG_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

int ensure_staging(hg_grid* g) {
    if (g->staging) return HG_OK;
    long long n = (long long)g->nx * g->ny * g->nz;
    long long ng = (long long)(g->nx + 2) * (g->ny + 2) * (g->nz + 2);
    long long want = 2 * n > ng ? 2 * n : ng;
    HG_CUDA(cudaMalloc(&g->staging, (size_t)want * sizeof(double)));
    return HG_OK;
}

void fill_ylm_norms(YlmNorm& N) {
    const double pi = 3.14159265358979323846;
    for (int q = 0; q < kMaxQ; ++q) {
        N.n[q] = 0.0;
        N.inv_lm[q] = 0.0;
    }
    for (int l = 0; l <= kMaxL; ++l)
        for (int m = 0; m <= l; ++m) {
            double ratio = 1.0;  // (l-m)!/(l+m)!
            for (int t = l - m + 1; t <= l + m; ++t) ratio /= (double)t;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * pi) * ratio);
            N.n[l * l + l + m] = m == 0 ? K : sqrt(2.0) * K;
            if (l > m) N.inv_lm[l * l + l + m] = 1.0 / (double)(l - m);
        }
}

static int dt_size(int dtype) { return dtype == HG_DT_F64 ? 8 : 4; }

// Robin coefficients of every face ghost: a = nu/mu and the radii r_g, r_i (FP64 grids), alpha = 1 - a and
// beta = a r_i/r_g in float (compensated float grids); rejects nu/mu > 1 (unstable upwind update)
static int build_robin(hg_grid* g) {
    long long n = g->F.off[6];
    std::vector<double> c((size_t)(3 * n));
    double worst = 0.0;
    for (long long t = 0; t < n; ++t) {
        int gc[3], ic[3];
        int f = face_cell(g->F, g->nx, g->ny, g->nz, t, gc, ic);
        if ((f == 4 && (g->ziface & 1)) || (f == 5 && (g->ziface & 2))) {  // a slab interface: never updated
            c[3 * t] = 0.0;
            c[3 * t + 1] = 1.0;
            c[3 * t + 2] = 1.0;
            continue;
        }
        double xg[3], xi[3];
        for (int a = 0; a < 3; ++a) {
            xg[a] = g->origin[a] + (gc[a] + 0.5) * g->h;
            xi[a] = g->origin[a] + (ic[a] + 0.5) * g->h;
        }
        double rg = sqrt(xg[0] * xg[0] + xg[1] * xg[1] + xg[2] * xg[2]);
        double ri = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
        double along = xg[f / 2] * ((f % 2) ? 1.0 : -1.0);  // x_g . n (outward normal)
        if (!(rg > 0.0) || !(along > 0.0))
            return fail(HG_ERR_CFL, "Robin boundary: ghost (%d,%d,%d) does not face away from the origin; the domain must "
                                    "surround the coordinate origin", gc[0], gc[1], gc[2]);
        double a = g->nu / (fabs(along) / rg);
        if (a > worst) worst = a;
        c[3 * t] = a;
        c[3 * t + 1] = rg;
        c[3 * t + 2] = ri;
    }
    if (worst > 1.0 + 1e-12)
        return fail(HG_ERR_CFL, "Robin boundary: nu/mu = %.6f > 1 at some ghost (reduce dt or centre the domain)", worst);
    HG_CUDA(cudaMalloc(&g->robin, c.size() * sizeof(double)));
    HG_CUDA(cudaMemcpy(g->robin, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<float2> c32((size_t)n);  // alpha = 1 - a, beta = a r_i / r_g
    for (long long t = 0; t < n; ++t)
        c32[t] = make_float2((float)(1.0 - c[3 * t]), (float)(c[3 * t] * c[3 * t + 2] / c[3 * t + 1]));
    HG_CUDA(cudaMalloc(&g->robin32, c32.size() * sizeof(float2)));
    HG_CUDA(cudaMemcpy(g->robin32, c32.data(), c32.size() * sizeof(float2), cudaMemcpyHostToDevice));
    return HG_OK;
}

extern "C" void hg_free(hg_grid* g);

static void release(hg_grid* g) {
    if (g->adj) hg_free(g->adj);
    void* ptrs[] = {g->phi[0], g->phi[1], g->lo[0], g->lo[1], g->dlt[0], g->dlt[1], g->rho, g->robin, g->robin32,
                    g->red, g->dres, g->staging, g->acc[0], g->acc[1], g->io_rho[0], g->io_rho[1], g->io_acc[0],
                    g->io_acc[1]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& slot : g->io_ev)
        for (cudaEvent_t ev : slot)
            if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : g->io_done)
        if (ev) cudaEventDestroy(ev);
    if (g->io_up) cudaStreamDestroy(g->io_up);
    if (g->io_down) cudaStreamDestroy(g->io_down);
    if (g->prof_ev) {
        for (int e = 0; e < 2 * kProfPairs; ++e) cudaEventDestroy(g->prof_ev[e]);
        delete[] g->prof_ev;
    }
}

int smem_attr_once(const void* fn, int bytes, unsigned long long* done) {
    int dev = 0;
    HG_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (*done & bit) return HG_OK;
    HG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    // the whole unified L1 / shared array as shared memory, so that the blocks the registers allow also fit
    HG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
    *done |= bit;
    return HG_OK;
}

int device_error(hg_grid* g) {
    int e = 0;
    HG_CUDA(cudaMemcpyAsync(&e, g->derr, sizeof e, cudaMemcpyDeviceToHost, g->stream));
    HG_CUDA(cudaStreamSynchronize(g->stream));
    if (!e) return HG_OK;
    HG_CUDA(cudaMemsetAsync(g->derr, 0, sizeof e, g->stream));
    if (e & 1)
        return fail(HG_ERR_TIMEOUT, "a bounded wait inside a sub-step kernel gave up (the results of that launch are "
                                    "not valid)");
    return fail(HG_ERR_BOUNDS, "a sub-step kernel computed a store index outside its array (debug build; the store "
                               "was skipped, the results are not valid)");
}

int prof_fold(hg_grid* g) {
    if (!g->prof_used) return HG_OK;
    HG_CUDA(cudaStreamSynchronize(g->stream));
    for (int p = 0; p < g->prof_used; ++p) {
        float ms = 0.f;
        HG_CUDA(cudaEventElapsedTime(&ms, g->prof_ev[2 * p], g->prof_ev[2 * p + 1]));
        g->prof_ms += ms;
    }
    g->prof_count += g->prof_used;
    g->prof_used = 0;
    return HG_OK;
}

int prof_begin(hg_grid* g) {
    if (!g->prof) return HG_OK;
    if (g->prof_used == kProfPairs) {
        int rc = prof_fold(g);
        if (rc) return rc;
    }
    HG_CUDA(cudaEventRecord(g->prof_ev[2 * g->prof_used], g->stream));
    return HG_OK;
}

int prof_end(hg_grid* g) {
    if (!g->prof) return HG_OK;
    HG_CUDA(cudaEventRecord(g->prof_ev[2 * g->prof_used + 1], g->stream));
    ++g->prof_used;
    return HG_OK;
}

static int check_grid(const hg_grid* g) {
    if (!g) return fail(HG_ERR_ARG, "null grid");
    cudaError_t e = cudaSetDevice(g->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return HG_OK;
}

}  // namespace hg

using namespace hg;

extern "C" {

const char* hg_last_error(void) { return g_last_error.c_str(); }

static int init_grid(hg_grid** out, int nx, int ny, int nz, double h, const double origin[3], double c_h, double G,
                     double dt, int precision, int bc, int lmax, void* cuda_stream, int ziface) {
    g_last_error.clear();
    if (!out) return fail(HG_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(HG_ERR_ARG, "grid sizes must be >= 1 (got %d %d %d)", nx, ny, nz);
    if ((long long)nx * ny * nz > (1LL << 34)) return fail(HG_ERR_ARG, "grid too large");
    if (!(h > 0.0) || !(c_h > 0.0) || !(dt > 0.0) || !isfinite(G) || !isfinite(h) || !isfinite(c_h) || !isfinite(dt))
        return fail(HG_ERR_ARG, "h, c_h and dt must be positive and finite, G finite");
    if (!origin || !isfinite(origin[0]) || !isfinite(origin[1]) || !isfinite(origin[2]))
        return fail(HG_ERR_ARG, "origin must be 3 finite values");
    if (precision != HG_PREC_F32K && precision != HG_PREC_F64) return fail(HG_ERR_ARG, "unknown precision %d", precision);
    if (bc < HG_BC_DIRICHLET_ANALYTIC || bc > HG_BC_PERIODIC) return fail(HG_ERR_ARG, "unknown boundary condition %d", bc);
    if (bc == HG_BC_DIRICHLET_MULTIPOLE && (lmax < 0 || lmax > HG_MAX_LMAX))
        return fail(HG_ERR_ARG, "lmax must be in 0..%d", HG_MAX_LMAX);
    double nu = c_h * dt / h;
    if (nu * sqrt(3.0) > 1.0 + 1e-12)
        return fail(HG_ERR_CFL, "nu sqrt(3) = %.6f > 1: the explicit scheme is unstable", nu * sqrt(3.0));

    hg_grid* g = new hg_grid;
    memset(g, 0, sizeof *g);
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->h = h;
    for (int a = 0; a < 3; ++a) g->origin[a] = origin[a];
    g->c = c_h;
    g->G = G;
    g->dt = dt;
    g->prec = precision;
    g->bc = bc;
    g->lmax = bc == HG_BC_DIRICHLET_MULTIPOLE ? lmax : 0;
    g->stream = (cudaStream_t)cuda_stream;
    g->nu = nu;
    g->nu2 = nu * nu;
    g->src = (c_h * dt) * (c_h * dt) * 4.0 * 3.14159265358979323846 * G;
    g->esize = precision == HG_PREC_F64 ? 8 : 4;
    g->L = make_layout(nx, ny, nz, g->esize);
    g->F = make_faces(nx, ny, nz);
    g->tdepth = 1;
    g->ziface = ziface;
    fill_ylm_norms(g->ylm);
    int rc = HG_OK;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "cudaGetDevice");
    }
    if (rc == HG_OK && (bc == HG_BC_DIRICHLET_ANALYTIC || bc == HG_BC_DIRICHLET_MULTIPOLE)) {
        for (long long t = 0; t < g->F.off[6] && rc == HG_OK; ++t) {
            int gc[3], ic[3];
            const int f = face_cell(g->F, nx, ny, nz, t, gc, ic);
            if ((f == 4 && (ziface & 1)) || (f == 5 && (ziface & 2))) continue;  // a slab interface: no boundary data
            double r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double x = origin[a] + (gc[a] + 0.5) * h;
                r2 += x * x;
            }
            if (!(r2 > 0.0)) rc = fail(HG_ERR_ARG, "a ghost cell centre sits at the expansion origin");
        }
    }
    if (rc == HG_OK && bc == HG_BC_ROBIN) rc = build_robin(g);
    const size_t bytes = (size_t)g->L.elems * g->esize;
    const size_t lo_bytes = (size_t)g->L.elems * sizeof(hg::lo_code);
    auto alloc = [&](void** p, size_t nb) {
        if (rc != HG_OK) return;
        cudaError_t e2 = cudaMalloc(p, nb);
        if (e2 != cudaSuccess) {
            rc = cuda_fail(e2, "cudaMalloc(state)");
            return;
        }
        e2 = cudaMemsetAsync(*p, 0, nb, g->stream);
        if (e2 != cudaSuccess) rc = cuda_fail(e2, "cudaMemsetAsync(state)");
    };
    alloc(&g->phi[0], bytes);
    alloc(&g->phi[1], bytes);
    alloc(&g->rho, bytes);
    if (precision == HG_PREC_F32K) {
        alloc(&g->lo[0], lo_bytes);  // 16-bit codes of the compensation
        alloc(&g->lo[1], lo_bytes);
        alloc(&g->dlt[0], bytes);
    }
    if (rc == HG_OK) {
        g->red_elems = reduction_scratch_elems();
        e = cudaMalloc(&g->red, (size_t)g->red_elems * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&g->dres, (kMaxQ + 2) * sizeof(double));
        if (e == cudaSuccess) e = cudaMemsetAsync(g->dres, 0, (kMaxQ + 2) * sizeof(double), g->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(reduction scratch)");
        g->dsum = g->dres + kMaxQ;
        g->derr = (int*)(g->dres + kMaxQ + 1);
    }
    if (rc == HG_OK) {
        e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (rc != HG_OK) {
        release(g);
        delete g;
        return rc;
    }
    *out = g;
    return HG_OK;
}

// density already on the device -> stored source, sum(rho) on the device, and for the Dirichlet modes the moments
// and boundary data; asynchronous except for the Dirichlet moments (read back to the host)
static int set_density_device(hg_grid* g, const void* src, int dtype) {
    int rc;
    if ((rc = prepare_source(g, src, dtype))) return rc;
    if (g->bc == HG_BC_DIRICHLET_ANALYTIC || g->bc == HG_BC_DIRICHLET_MULTIPOLE) {
        if ((rc = compute_moments(g, src, dtype))) return rc;
        if ((rc = set_ghosts_dirichlet(g))) return rc;
    }
    return HG_OK;
}

int hg_init_grid(hg_grid** out, int nx, int ny, int nz, double h, const double origin[3], double c_h, double G,
                 double dt, int precision, int bc, int lmax, void* cuda_stream) {
    HG_RANGE("hg_init_grid");
    return init_grid(out, nx, ny, nz, h, origin, c_h, G, dt, precision, bc, lmax, cuda_stream, 0);
}

int hg_init_slab(hg_grid** out, int nx, int ny, int nz, double h, const double origin[3], double c_h, double G,
                 double dt, int precision, int bc, int lmax, void* cuda_stream, int z_interfaces) {
    HG_RANGE("hg_init_slab");
    if (z_interfaces < 0 || z_interfaces > 3) return fail(HG_ERR_ARG, "z_interfaces must be 0..3");
    if (z_interfaces && bc == HG_BC_PERIODIC)
        return fail(HG_ERR_STATE, "slab interfaces are built for the Robin and Dirichlet boundaries (a periodic "
                                  "source needs the mean density of the whole grid)");
    return init_grid(out, nx, ny, nz, h, origin, c_h, G, dt, precision, bc, lmax, cuda_stream, z_interfaces);
}

int hg_set_density(hg_grid* g, const void* rho, int dtype, int on_device) {
    HG_RANGE("hg_set_density");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!rho) return fail(HG_ERR_ARG, "null density");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    const long long n = (long long)g->nx * g->ny * g->nz;
    const void* src = rho;
    if (!on_device) {
        if ((rc = ensure_staging(g))) return rc;
        HG_CUDA(cudaMemcpyAsync(g->staging, rho, (size_t)n * dt_size(dtype), cudaMemcpyHostToDevice, g->stream));
        src = g->staging;
    }
    if ((rc = set_density_device(g, src, dtype))) return rc;
    if (!on_device) HG_CUDA(cudaStreamSynchronize(g->stream));  // the staging buffer is reused by later calls
    return HG_OK;
}

int hg_set_phi(hg_grid* g, const void* phi, const void* phi_prev, int dtype, int on_device) {
    HG_RANGE("hg_set_phi");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!phi) return fail(HG_ERR_ARG, "null phi");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    const long long n = (long long)g->nx * g->ny * g->nz;
    const void* a = phi;
    const void* b = phi_prev;
    if (!on_device) {
        if ((rc = ensure_staging(g))) return rc;
        size_t bytes = (size_t)n * dt_size(dtype);
        HG_CUDA(cudaMemcpyAsync(g->staging, phi, bytes, cudaMemcpyHostToDevice, g->stream));
        a = g->staging;
        if (phi_prev) {
            HG_CUDA(cudaMemcpyAsync((char*)g->staging + bytes, phi_prev, bytes, cudaMemcpyHostToDevice, g->stream));
            b = (const char*)g->staging + bytes;
        }
    }
    if ((rc = set_phi_device(g, a, b, dtype))) return rc;
    if ((rc = seed_ghosts(g))) return rc;
    g->step = 0;
    if (!on_device) HG_CUDA(cudaStreamSynchronize(g->stream));
    return HG_OK;
}

int hg_set_temporal_depth(hg_grid* g, int k) {
    HG_RANGE("hg_set_temporal_depth");
    int rc = check_grid(g);
    if (rc) return rc;
    if (k < 1 || k > HG_MAX_TEMPORAL_DEPTH)
        return fail(HG_ERR_ARG, "temporal depth must be in 1..%d", HG_MAX_TEMPORAL_DEPTH);
    if (k > 1 && g->ziface)
        return fail(HG_ERR_STATE, "a slab exchanges its interface planes before every sub-step: temporal depth 1 only");
    if (k > 1 && g->prec != HG_PREC_F32K)
        return fail(HG_ERR_ARG, "temporal blocking is built for HG_PREC_F32K only (FP64 sub-steps are bound by the "
                                "FP64 and integer pipes, at 22-41%% of HBM bandwidth, so fusing them saves nothing)");
    if (k > 1 && !g->dlt[1]) {
        size_t bytes = (size_t)g->L.elems * g->esize;
        HG_CUDA(cudaMalloc(&g->dlt[1], bytes));
        HG_CUDA(cudaMemsetAsync(g->dlt[1], 0, bytes, g->stream));
    }
    g->tdepth = k;
    return HG_OK;
}

int hg_set_temporal_exact(hg_grid* g, int exact) {
    HG_RANGE("hg_set_temporal_exact");
    int rc = check_grid(g);
    if (rc) return rc;
    g->texact = exact ? 1 : 0;
    return HG_OK;
}

int hg_set_block_depth(hg_grid* g, int planes) {
    HG_RANGE("hg_set_block_depth");
    int rc = check_grid(g);
    if (rc) return rc;
    if (planes < 0) return fail(HG_ERR_ARG, "planes must be >= 0");
    g->zb = planes;
    return HG_OK;
}

int hg_step(hg_grid* g, int n_substeps) {
    HG_RANGE("hg_step");
    int rc = check_grid(g);
    if (rc) return rc;
    if (n_substeps < 0) return fail(HG_ERR_ARG, "n_substeps must be >= 0");
    int s = 0;
    while (s < n_substeps) {
        int k = n_substeps - s < g->tdepth ? n_substeps - s : g->tdepth;
        // the sweep launches also write the face ghosts of the new level (Robin update, periodic copy)
        if (k >= 2) {
            if ((rc = launch_temporal(g, k))) return rc;
        } else {
            if ((rc = launch_step_single(g))) return rc;
        }
        g->cur = 1 - g->cur;
        if (k >= 2) g->dcur = 1 - g->dcur;
        s += k;
        g->step += k;
    }
    return HG_OK;
}

int hg_accel(hg_grid* g, void* ax, void* ay, void* az, int dtype) {
    HG_RANGE("hg_accel");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!ax || !ay || !az) return fail(HG_ERR_ARG, "null acceleration buffer");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    return accel(g, ax, ay, az, dtype);
}

int hg_get_phi(hg_grid* g, void* out, int dtype, int on_device) {
    HG_RANGE("hg_get_phi");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!out) return fail(HG_ERR_ARG, "null output");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    if (on_device) return unpack_phi(g, out, dtype);
    if ((rc = ensure_staging(g))) return rc;
    if ((rc = unpack_phi(g, g->staging, dtype))) return rc;
    size_t bytes = (size_t)g->nx * g->ny * g->nz * dt_size(dtype);
    HG_CUDA(cudaMemcpyAsync(out, g->staging, bytes, cudaMemcpyDeviceToHost, g->stream));
    HG_CUDA(cudaStreamSynchronize(g->stream));
    return HG_OK;
}

int hg_get_phi_ghosted(hg_grid* g, double* out) {
    HG_RANGE("hg_get_phi_ghosted");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!out) return fail(HG_ERR_ARG, "null output");
    if ((rc = ensure_staging(g))) return rc;
    if ((rc = unpack_phi_ghosted(g, g->staging))) return rc;
    size_t bytes = (size_t)(g->nx + 2) * (g->ny + 2) * (g->nz + 2) * sizeof(double);
    HG_CUDA(cudaMemcpyAsync(out, g->staging, bytes, cudaMemcpyDeviceToHost, g->stream));
    HG_CUDA(cudaStreamSynchronize(g->stream));
    return HG_OK;
}

int hg_get_stats(hg_grid* g, hg_stats* s) {
    HG_RANGE("hg_get_stats");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!s) return fail(HG_ERR_ARG, "null stats");
    if ((rc = stats(g, s))) return rc;
    if (s->nonfinite) return fail(HG_ERR_NONFINITE, "non-finite values in the state after %lld sub-steps", s->step);
    return HG_OK;
}

int hg_get_moments(hg_grid* g, double* Q) {
    HG_RANGE("hg_get_moments");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!Q) return fail(HG_ERR_ARG, "null output");
    if (!(g->bc == HG_BC_DIRICHLET_ANALYTIC || g->bc == HG_BC_DIRICHLET_MULTIPOLE) || !g->have_Q)
        return fail(HG_ERR_STATE, "moments exist only for the Dirichlet modes after hg_set_density");
    int nq = (g->lmax + 1) * (g->lmax + 1);
    for (int q = 0; q < nq; ++q) Q[q] = g->Q[q];
    return HG_OK;
}

// ---- slab decomposition along z (one grid split over several grids, one per device or process) ----
int hg_set_z_interface(hg_grid* g, int lo, int hi) {
    HG_RANGE("hg_set_z_interface");
    int rc = check_grid(g);
    if (rc) return rc;
    if ((lo || hi) && g->bc == HG_BC_PERIODIC)
        return fail(HG_ERR_STATE, "slab interfaces are built for the Robin and Dirichlet boundaries (a periodic "
                                  "source needs the mean density of the whole grid)");
    if ((lo || hi) && g->tdepth > 1)
        return fail(HG_ERR_STATE, "a slab exchanges its interface planes before every sub-step: temporal depth 1 only");
    g->ziface = (lo ? 1 : 0) | (hi ? 2 : 0);
    return HG_OK;
}

size_t hg_plane_bytes(const hg_grid* g) {
    HG_RANGE("hg_plane_bytes");
    if (!g) return 0;
    const size_t n = (size_t)g->nx * g->ny;
    return g->prec == HG_PREC_F64 ? n * sizeof(double) : n * (sizeof(float) + sizeof(lo_code));
}

// one z-plane k of phi^n between the padded state and a packed buffer (F64: nx*ny doubles; F32K: nx*ny floats, then
// nx*ny compensation codes), with 2-D copies on the grid's stream
static int plane_copy(hg_grid* g, int k, void* buf, int on_device, bool to_state) {
    const int c = g->cur;
    const size_t n = (size_t)g->nx * g->ny;
    const Layout& L = g->L;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                          : (to_state ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    char* b = (char*)buf;
    const size_t es = (size_t)g->esize;
    char* hi = (char*)g->phi[c] + (size_t)L.at(0, 0, k) * es;
    if (to_state)
        HG_CUDA(cudaMemcpy2DAsync(hi, L.pitch * es, b, g->nx * es, g->nx * es, g->ny, kind, g->stream));
    else
        HG_CUDA(cudaMemcpy2DAsync(b, g->nx * es, hi, L.pitch * es, g->nx * es, g->ny, kind, g->stream));
    if (g->prec == HG_PREC_F32K) {
        const size_t ls = sizeof(lo_code);
        char* lo = (char*)g->lo[c] + (size_t)L.at(0, 0, k) * ls;
        char* bl = b + n * es;
        if (to_state)
            HG_CUDA(cudaMemcpy2DAsync(lo, L.pitch * ls, bl, g->nx * ls, g->nx * ls, g->ny, kind, g->stream));
        else
            HG_CUDA(cudaMemcpy2DAsync(bl, g->nx * ls, lo, L.pitch * ls, g->nx * ls, g->ny, kind, g->stream));
    }
    if (!on_device) HG_CUDA(cudaStreamSynchronize(g->stream));
    return HG_OK;
}

int hg_get_plane(hg_grid* g, int which, void* buf, int on_device) {
    HG_RANGE("hg_get_plane");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!buf || (which != 0 && which != 1)) return fail(HG_ERR_ARG, "null buffer, or which not 0 or 1");
    return plane_copy(g, which ? g->nz - 1 : 0, buf, on_device, false);
}

int hg_put_ghost_plane(hg_grid* g, int side, const void* buf, int on_device) {
    HG_RANGE("hg_put_ghost_plane");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!buf || (side != 0 && side != 1)) return fail(HG_ERR_ARG, "null buffer, or side not 0 or 1");
    if (!(g->ziface & (1 << side))) return fail(HG_ERR_STATE, "that z face is not a slab interface");
    return plane_copy(g, side ? g->nz : -1, const_cast<void*>(buf), on_device, true);
}

int hg_set_boundary_moments(hg_grid* g, const double* Q) {
    HG_RANGE("hg_set_boundary_moments");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!Q) return fail(HG_ERR_ARG, "null moments");
    if (!(g->bc == HG_BC_DIRICHLET_ANALYTIC || g->bc == HG_BC_DIRICHLET_MULTIPOLE))
        return fail(HG_ERR_STATE, "boundary moments exist only for the Dirichlet modes");
    const int nq = (g->lmax + 1) * (g->lmax + 1);
    for (int q = 0; q < kMaxQ; ++q) g->Q[q] = q < nq ? Q[q] : 0.0;
    g->have_Q = 1;
    return set_ghosts_dirichlet(g);
}

int hg_compare(hg_grid* g, const double* phi_P, int on_device, double out[3]) {
    HG_RANGE("hg_compare");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!phi_P || !out) return fail(HG_ERR_ARG, "null argument");
    const double* P = phi_P;
    if (!on_device) {
        if ((rc = ensure_staging(g))) return rc;
        HG_CUDA(cudaMemcpyAsync(g->staging, phi_P, (size_t)g->nx * g->ny * g->nz * sizeof(double),
                                cudaMemcpyHostToDevice, g->stream));
        P = g->staging;
    }
    return compare(g, P, out);
}

// ---- checkpoint / resume ----
// The stored source s = (c_h dt)^2 4 pi G (rho - rho_bar), the Dirichlet ghosts (functions of h, the origin and G)
// and the Robin coefficients (functions of nu = c_h dt / h and the geometry) are only valid for the grid that wrote
// them, so the header records every parameter they depend on and a load accepts only a bit-identical match.
struct StateHeader {
    char magic[8];
    int nx, ny, nz, prec, bc, lmax, cur, have_Q;
    long long step;
    double mass, rho_bar;
    double h, origin[3], c, G, dt;
    double Q[kMaxQ];
};

static bool same_bits(double a, double b) { return memcmp(&a, &b, sizeof a) == 0; }

static int n_buffers(const hg_grid* g) { return g->prec == HG_PREC_F64 ? 3 : 6; }
static void** buffer(hg_grid* g, int b) {
    void** all[6] = {&g->phi[0], &g->phi[1], &g->rho, &g->lo[0], &g->lo[1], &g->dlt[g->dcur]};
    return all[b];
}
static size_t buffer_bytes(const hg_grid* g, int b) {
    return (size_t)g->L.elems * (b == 3 || b == 4 ? sizeof(lo_code) : (size_t)g->esize);
}

size_t hg_state_bytes(const hg_grid* g) {
    HG_RANGE("hg_state_bytes");
    if (!g) return 0;
    size_t n = sizeof(StateHeader);
    for (int b = 0; b < n_buffers(g); ++b) n += buffer_bytes(g, b);
    return n;
}

int hg_save_state(hg_grid* g, void* buf, int on_device) {
    HG_RANGE("hg_save_state");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!buf) return fail(HG_ERR_ARG, "null buffer");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    StateHeader H;
    memset(&H, 0, sizeof H);
    memcpy(H.magic, "HGSTATE2", 8);
    H.nx = g->nx;
    H.ny = g->ny;
    H.nz = g->nz;
    H.prec = g->prec;
    H.bc = g->bc;
    H.lmax = g->lmax;
    H.cur = g->cur;
    H.have_Q = g->have_Q;
    H.step = g->step;
    H.h = g->h;
    for (int a = 0; a < 3; ++a) H.origin[a] = g->origin[a];
    H.c = g->c;
    H.G = g->G;
    H.dt = g->dt;
    if ((rc = sync_mass(g))) return rc;
    H.mass = g->mass;
    H.rho_bar = g->rho_bar;
    memcpy(H.Q, g->Q, sizeof H.Q);
    if (on_device)
        HG_CUDA(cudaMemcpyAsync(buf, &H, sizeof H, cudaMemcpyHostToDevice, g->stream));
    else
        memcpy(buf, &H, sizeof H);
    char* p = (char*)buf + sizeof H;
    for (int b = 0; b < n_buffers(g); ++b) {
        HG_CUDA(cudaMemcpyAsync(p, *buffer(g, b), buffer_bytes(g, b), kind, g->stream));
        p += buffer_bytes(g, b);
    }
    HG_CUDA(cudaStreamSynchronize(g->stream));  // the header copy reads a stack variable
    return HG_OK;
}

int hg_load_state(hg_grid* g, const void* buf, int on_device) {
    HG_RANGE("hg_load_state");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!buf) return fail(HG_ERR_ARG, "null buffer");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    StateHeader H;
    if (on_device) {
        HG_CUDA(cudaMemcpyAsync(&H, buf, sizeof H, cudaMemcpyDeviceToHost, g->stream));
        HG_CUDA(cudaStreamSynchronize(g->stream));
    } else {
        memcpy(&H, buf, sizeof H);
    }
    if (memcmp(H.magic, "HGSTATE2", 8) != 0 || H.nx != g->nx || H.ny != g->ny || H.nz != g->nz || H.prec != g->prec ||
        H.bc != g->bc || H.lmax != g->lmax)
        return fail(HG_ERR_ARG, "state buffer does not match this grid");
    if (!same_bits(H.h, g->h) || !same_bits(H.origin[0], g->origin[0]) || !same_bits(H.origin[1], g->origin[1]) ||
        !same_bits(H.origin[2], g->origin[2]) || !same_bits(H.c, g->c) || !same_bits(H.G, g->G) ||
        !same_bits(H.dt, g->dt))
        return fail(HG_ERR_ARG, "state buffer was written by a grid with another h, origin, c_h, G or dt");
    const char* p = (const char*)buf + sizeof H;
    for (int b = 0; b < n_buffers(g); ++b) {
        HG_CUDA(cudaMemcpyAsync(*buffer(g, b), p, buffer_bytes(g, b), kind, g->stream));
        p += buffer_bytes(g, b);
    }
    if (!on_device) HG_CUDA(cudaStreamSynchronize(g->stream));
    g->cur = H.cur;
    g->have_Q = H.have_Q;
    g->step = H.step;
    g->mass = H.mass;
    g->rho_bar = H.rho_bar;
    g->mass_pending = 0;
    memcpy(g->Q, H.Q, sizeof H.Q);
    return HG_OK;
}

int hg_profile(hg_grid* g, int enable) {
    HG_RANGE("hg_profile");
    int rc = check_grid(g);
    if (rc) return rc;
    if (enable && !g->prof_ev) {
        g->prof_ev = new cudaEvent_t[2 * kProfPairs];
        for (int e = 0; e < 2 * kProfPairs; ++e) HG_CUDA(cudaEventCreate(&g->prof_ev[e]));
    }
    if (!enable && (rc = prof_fold(g))) return rc;
    g->prof = enable ? 1 : 0;
    return HG_OK;
}

int hg_profile_read(hg_grid* g, double* substep_kernel_ms, long long* substep_launches, long long* kernel_launches) {
    HG_RANGE("hg_profile_read");
    int rc = check_grid(g);
    if (rc) return rc;
    if ((rc = prof_fold(g))) return rc;
    if (substep_kernel_ms) *substep_kernel_ms = g->prof_ms;
    if (substep_launches) *substep_launches = g->prof_count;
    if (kernel_launches) *kernel_launches = g->launches;
    g->prof_ms = 0.0;
    g->prof_count = 0;
    return HG_OK;
}

// ---- adjoint ----
int hg_adjoint_reset(hg_grid* g) {
    HG_RANGE("hg_adjoint_reset");
    int rc = check_grid(g);
    if (rc) return rc;
    if (g->ziface) return fail(HG_ERR_STATE, "the adjoint is built for whole grids, not for slabs");
    if (!g->adj) {
        // Dirichlet data do not depend on rho in the adjoint: the shadow grid keeps zero boundary data (no density is
        // ever set on it, so its source is zero as well)
        const int bc = (g->bc == HG_BC_DIRICHLET_MULTIPOLE) ? HG_BC_DIRICHLET_ANALYTIC : g->bc;
        if ((rc = hg_init_grid(&g->adj, g->nx, g->ny, g->nz, g->h, g->origin, g->c, g->G, g->dt, g->prec, bc, 0,
                               g->stream)))
            return rc;
        const size_t bytes = (size_t)g->L.elems * g->esize;
        HG_CUDA(cudaMalloc(&g->acc[0], bytes));
        if (g->prec == HG_PREC_F32K) HG_CUDA(cudaMalloc(&g->acc[1], bytes));
    }
    hg_grid* a = g->adj;
    const size_t bytes = (size_t)a->L.elems * a->esize, lo_bytes = (size_t)a->L.elems * sizeof(lo_code);
    void* bufs[] = {a->phi[0], a->phi[1], a->dlt[0], a->dlt[1], g->acc[0], g->acc[1]};
    for (void* b : bufs)
        if (b) HG_CUDA(cudaMemsetAsync(b, 0, bytes, g->stream));
    for (void* b : {a->lo[0], a->lo[1]})
        if (b) HG_CUDA(cudaMemsetAsync(b, 0, lo_bytes, g->stream));
    a->cur = 0;
    a->dcur = 0;
    a->step = 0;
    return HG_OK;
}

int hg_adjoint_inject(hg_grid* g, const void* dL_dphi, int dtype, int on_device) {
    HG_RANGE("hg_adjoint_inject");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!g->adj) return fail(HG_ERR_STATE, "call hg_adjoint_reset first");
    if (!dL_dphi) return fail(HG_ERR_ARG, "null input");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    hg_grid* a = g->adj;
    const void* v = dL_dphi;
    if (!on_device) {
        if ((rc = ensure_staging(a))) return rc;
        HG_CUDA(cudaMemcpyAsync(a->staging, dL_dphi, (size_t)a->nx * a->ny * a->nz * dt_size(dtype),
                                cudaMemcpyHostToDevice, a->stream));
        v = a->staging;
    }
    if ((rc = adjoint_inject(a, v, dtype))) return rc;
    // the ghosts of a periodic level are copies of its interior, so they follow the injection
    if (a->bc == HG_BC_PERIODIC && (rc = launch_periodic_fill(a, a->cur))) return rc;
    if (!on_device) HG_CUDA(cudaStreamSynchronize(a->stream));
    return HG_OK;
}

int hg_adjoint_step(hg_grid* g, int n_substeps) {
    HG_RANGE("hg_adjoint_step");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!g->adj) return fail(HG_ERR_STATE, "call hg_adjoint_reset first");
    if (n_substeps < 0) return fail(HG_ERR_ARG, "n_substeps must be >= 0");
    hg_grid* a = g->adj;
    for (int s = 0; s < n_substeps; ++s) {
        if ((rc = adjoint_accumulate(a, g->acc[0], g->acc[1]))) return rc;
        if ((rc = launch_step_single(a))) return rc;
        a->cur = 1 - a->cur;
        ++a->step;
    }
    return HG_OK;
}

int hg_adjoint_grad(hg_grid* g, void* dL_drho, int dtype, int on_device) {
    HG_RANGE("hg_adjoint_grad");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!g->adj) return fail(HG_ERR_STATE, "call hg_adjoint_reset first");
    if (!dL_drho) return fail(HG_ERR_ARG, "null output");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    hg_grid* a = g->adj;
    if (on_device) return adjoint_gradient(a, g->acc[0], g->acc[1], dL_drho, dtype, a->red);
    if ((rc = ensure_staging(a))) return rc;
    if ((rc = adjoint_gradient(a, g->acc[0], g->acc[1], a->staging, dtype, a->red))) return rc;
    HG_CUDA(cudaMemcpyAsync(dL_drho, a->staging, (size_t)a->nx * a->ny * a->nz * dt_size(dtype),
                            cudaMemcpyDeviceToHost, a->stream));
    HG_CUDA(cudaStreamSynchronize(a->stream));
    return HG_OK;
}

// ---- host I/O pipeline ----
static size_t align_up(size_t b, size_t a) { return (b + a - 1) / a * a; }

static int io_ready(hg_grid* g, size_t rho_bytes, size_t acc_bytes) {
    if (!g->io_up) {
        HG_CUDA(cudaStreamCreateWithFlags(&g->io_up, cudaStreamNonBlocking));
        HG_CUDA(cudaStreamCreateWithFlags(&g->io_down, cudaStreamNonBlocking));
        for (auto& slot : g->io_ev)
            for (cudaEvent_t& ev : slot) HG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        for (cudaEvent_t& ev : g->io_done) HG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    if (rho_bytes <= g->io_rho_bytes && acc_bytes <= g->io_acc_bytes) return HG_OK;
    // the slots grow (a wider dtype) only while nothing of the pipeline is in flight
    HG_CUDA(cudaStreamSynchronize(g->stream));
    HG_CUDA(cudaStreamSynchronize(g->io_up));
    HG_CUDA(cudaStreamSynchronize(g->io_down));
    if (rho_bytes > g->io_rho_bytes) {
        for (void*& p : g->io_rho) {
            if (p) HG_CUDA(cudaFree(p));
            p = nullptr;
        }
        g->io_rho_bytes = 0;
        for (void*& p : g->io_rho) HG_CUDA(cudaMalloc(&p, rho_bytes));
        g->io_rho_bytes = rho_bytes;
    }
    if (acc_bytes > g->io_acc_bytes) {
        for (void*& p : g->io_acc) {
            if (p) HG_CUDA(cudaFree(p));
            p = nullptr;
        }
        g->io_acc_bytes = 0;
        for (void*& p : g->io_acc) HG_CUDA(cudaMalloc(&p, acc_bytes));
        g->io_acc_bytes = acc_bytes;
    }
    return HG_OK;
}

int hg_adjoint(hg_grid* g, const void* dL_dphiT, int T, void* dL_drho, int dtype, int on_device) {
    HG_RANGE("hg_adjoint");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!dL_dphiT || !dL_drho) return fail(HG_ERR_ARG, "null adjoint buffer");
    if (T < 0) return fail(HG_ERR_ARG, "T must be >= 0");
    if ((rc = hg_adjoint_reset(g))) return rc;
    if ((rc = hg_adjoint_inject(g, dL_dphiT, dtype, on_device))) return rc;
    if ((rc = hg_adjoint_step(g, T))) return rc;
    return hg_adjoint_grad(g, dL_drho, dtype, on_device);
}

int hg_io_step(hg_grid* g, const void* rho_host, int rho_dtype, int n_substeps, void* ax_host, void* ay_host,
               void* az_host, int acc_dtype) {
    HG_RANGE("hg_io_step");
    int rc = check_grid(g);
    if (rc) return rc;
    if (n_substeps < 0) return fail(HG_ERR_ARG, "n_substeps must be >= 0");
    const bool want_acc = ax_host || ay_host || az_host;
    if (want_acc && !(ax_host && ay_host && az_host)) return fail(HG_ERR_ARG, "give all three acceleration buffers");
    if (rho_host && rho_dtype != HG_DT_F32 && rho_dtype != HG_DT_F64)
        return fail(HG_ERR_ARG, "unknown density dtype %d", rho_dtype);
    if (want_acc && acc_dtype != HG_DT_F32 && acc_dtype != HG_DT_F64)
        return fail(HG_ERR_ARG, "unknown acceleration dtype %d", acc_dtype);
    const size_t n = (size_t)g->nx * g->ny * g->nz;
    const size_t rho_bytes = rho_host ? n * dt_size(rho_dtype) : 0;
    const size_t comp = want_acc ? align_up(n * dt_size(acc_dtype), 256) : 0;  // one component, 256-byte aligned
    if ((rc = io_ready(g, rho_bytes, 3 * comp))) return rc;
    const int k = (int)(g->io_issued & 1);
    cudaEvent_t* ev = g->io_ev[k];  // 0 uploaded, 1 consumed, 2 acceleration written
    constexpr int kRing = (int)(sizeof g->io_done / sizeof g->io_done[0]);
    cudaEvent_t done = g->io_done[g->io_issued % kRing];
    cudaEvent_t prev_done = g->io_done[(g->io_issued + kRing - 2) % kRing];  // this slot's previous user, if any
    if (rho_host) {
        HG_CUDA(cudaStreamWaitEvent(g->io_up, ev[1], 0));  // the slot's previous density has been packed
        HG_CUDA(cudaMemcpyAsync(g->io_rho[k], rho_host, rho_bytes, cudaMemcpyHostToDevice, g->io_up));
        HG_CUDA(cudaEventRecord(ev[0], g->io_up));
        HG_CUDA(cudaStreamWaitEvent(g->stream, ev[0], 0));
        if ((rc = set_density_device(g, g->io_rho[k], rho_dtype))) return rc;
        HG_CUDA(cudaEventRecord(ev[1], g->stream));
    }
    if ((rc = hg_step(g, n_substeps))) return rc;
    char* a = (char*)g->io_acc[k];
    if (want_acc) {
        if (g->io_issued >= 2)  // the slot's previous acceleration has been downloaded
            HG_CUDA(cudaStreamWaitEvent(g->stream, prev_done, 0));
        if ((rc = accel(g, a, a + comp, a + 2 * comp, acc_dtype))) return rc;
    }
    HG_CUDA(cudaEventRecord(ev[2], g->stream));
    HG_CUDA(cudaStreamWaitEvent(g->io_down, ev[2], 0));
    if (want_acc) {
        const size_t bytes = n * dt_size(acc_dtype);
        HG_CUDA(cudaMemcpyAsync(ax_host, a, bytes, cudaMemcpyDeviceToHost, g->io_down));
        HG_CUDA(cudaMemcpyAsync(ay_host, a + comp, bytes, cudaMemcpyDeviceToHost, g->io_down));
        HG_CUDA(cudaMemcpyAsync(az_host, a + 2 * comp, bytes, cudaMemcpyDeviceToHost, g->io_down));
    }
    HG_CUDA(cudaEventRecord(done, g->io_down));
    ++g->io_issued;
    return HG_OK;
}

int hg_io_wait(hg_grid* g, int keep) {
    HG_RANGE("hg_io_wait");
    int rc = check_grid(g);
    if (rc) return rc;
    if (keep < 0) return fail(HG_ERR_ARG, "keep must be >= 0");
    // completion events form a ring of 8: exact for the last 8 calls, conservative (waits longer) for older ones
    constexpr int kRing = (int)(sizeof g->io_done / sizeof g->io_done[0]);
    while (g->io_waited < g->io_issued - keep) {
        HG_CUDA(cudaEventSynchronize(g->io_done[g->io_waited % kRing]));
        ++g->io_waited;
    }
    return HG_OK;
}

int hg_check_bounded_wait(hg_grid* g) {
    HG_RANGE("hg_check_bounded_wait");
    int rc = check_grid(g);
    if (rc) return rc;
    if ((rc = device_error(g))) return rc;  // an earlier error is reported as such, not taken for the self-test's
    rc = wait_selftest(g);
    if (rc == HG_ERR_TIMEOUT) return HG_OK;  // the wait gave up and the host saw it
    if (rc == HG_OK) return fail(HG_ERR_STATE, "the bounded-wait self-test did not report its timeout");
    return rc;
}

int hg_is_debug_build(void) { return kDebugChecks ? 1 : 0; }

int hg_check_bounds(hg_grid* g) {
    HG_RANGE("hg_check_bounds");
    int rc = check_grid(g);
    if (rc) return rc;
    if (!kDebugChecks) return fail(HG_ERR_STATE, "a release build has no index checks");
    if ((rc = device_error(g))) return rc;
    if ((rc = bounds_selftest(g))) return rc;
    rc = device_error(g);
    if (rc == HG_ERR_BOUNDS) return HG_OK;
    if (rc == HG_OK) return fail(HG_ERR_STATE, "the index check did not report the index past the array");
    return rc;
}

int hg_sync(hg_grid* g) {
    HG_RANGE("hg_sync");
    int rc = check_grid(g);
    if (rc) return rc;
    HG_CUDA(cudaStreamSynchronize(g->stream));
    if ((rc = device_error(g))) return rc;
    if (g->io_up) {
        HG_CUDA(cudaStreamSynchronize(g->io_up));
        HG_CUDA(cudaStreamSynchronize(g->io_down));
        g->io_waited = g->io_issued;
    }
    HG_CUDA(cudaGetLastError());
    return HG_OK;
}

void hg_free(hg_grid* g) {
    HG_RANGE("hg_free");
    if (!g) return;
    cudaSetDevice(g->device);
    cudaStreamSynchronize(g->stream);
    if (g->io_up) cudaStreamSynchronize(g->io_up);
    if (g->io_down) cudaStreamSynchronize(g->io_down);
    release(g);
    delete g;
}

}  // extern "C"
