// Discrete adjoint of the sub-stepping, for gradients dL/drho through T sub-steps (the differentiation workload;
// the paper itself has no adjoint: this is the transpose of its Eq. HNeq. time-stepper, Sec. 2).
//
// The sub-step is linear in (phi^n, phi^{n-1}, s).  Writing its transpose in gather form gives, for the adjoint
// variables lambda^m = dL/dphi^m (interior cells) and the Robin ghost variables,
//   lambda_c^m = 2 lambda_c^{m+1} - lambda_c^{m+2} + nu^2 sum_{6 nb}(mu_nb^{m+1} - lambda_c^{m+1}) + injection,
//   mu_g^m     = alpha_g mu_g^{m+1} + beta_g lambda_i^{m+1}                              (Robin ghosts),
// where mu_nb is lambda_nb for an interior neighbour, 0 for a Dirichlet ghost (boundary data do not depend on rho),
// the wrapped value for a periodic ghost, and mu_g = (beta_g / nu^2) dL/dphi_g for a Robin ghost.  With that scaling
// the recursion is exactly the forward sub-step with a zero source, so the adjoint runs on the same kernels, in a
// shadow grid of the same geometry, precision and boundary condition whose boundary data are zero.
// Then dL/ds_c = -sum_{m=1..T} lambda_c^m and dL/drho = (c dt)^2 4 pi G dL/ds (minus its mean for periodic
// boundaries, the transpose of rho -> rho - mean(rho)).  The recursion needs no forward states.
//
// Kernels here: add an injection into the shadow state, accumulate sum_m lambda^m (float pairs for the compensated
// precision, double for FP64), and turn the sum into the gradient.
#include "cell.cuh"
#include "hg_internal.cuh"

namespace hg {

namespace {

constexpr int kThreads = 256;

template <class F>
__device__ __forceinline__ void for_cells(const Layout& L, F&& f) {
    const long long rows = (long long)L.ny * L.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = (int)(row % L.ny), k = (int)(row / L.ny);
        const long long base = row * L.nx;
        for (int i = threadIdx.x; i < L.nx; i += blockDim.x) f(L.at(i, j, k), base + i);
    }
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// lambda^m += v on the interior; for the compensated state the increment dlt = lambda^m - lambda^{m+1} moves too
__global__ void k_inject(int prec, const void* v, int vdt, void* hi, void* lo, void* dlt, Layout L) {
    for_cells(L, [&](long long q, long long c) {
        const double x = vdt == HG_DT_F64 ? ((const double*)v)[c] : (double)((const float*)v)[c];
        if (prec == HG_PREC_F64) {
            ((double*)hi)[q] += x;
        } else {
            float* h = (float*)hi;
            lo_t* l = (lo_t*)lo;
            const float xh = (float)x, xl = (float)(x - (double)xh);
            const float h0 = h[q];
            float s, e;
            two_sum(h0, xh, s, e);
            const float t = (lo_decode(h0, l[q]) + xl) + e;
            const float hn = s + t;
            h[q] = hn;
            l[q] = lo_encode(hn, t - (hn - s));
            ((float*)dlt)[q] += xh;
        }
    });
}

// acc += lambda^m on the interior
__global__ void k_accumulate(int prec, const void* hi, const void* lo, void* acc_a, void* acc_b, Layout L) {
    for_cells(L, [&](long long q, long long) {
        if (prec == HG_PREC_F64) {
            ((double*)acc_a)[q] += ((const double*)hi)[q];
        } else {
            float* a = (float*)acc_a;
            float* b = (float*)acc_b;
            float s, e;
            const float h = ((const float*)hi)[q];
            two_sum(a[q], h, s, e);
            const float t = b[q] + (e + lo_decode(h, ((const lo_t*)lo)[q]));
            a[q] = s + t;
            b[q] = t - (a[q] - s);
        }
    });
}

// out = scale * acc - shift (dense, dtype); with want_sum the same pass leaves per-block partial sums of scale*acc
__global__ void __launch_bounds__(kThreads) k_grad(int prec, const void* acc_a, const void* acc_b, void* out, int odt,
                                                   Layout L, double scale, double shift, double* partial) {
    __shared__ double sh[32];
    double sum = 0.0;
    for_cells(L, [&](long long q, long long c) {
        const double a = prec == HG_PREC_F64 ? ((const double*)acc_a)[q]
                                             : (double)((const float*)acc_a)[q] + (double)((const float*)acc_b)[q];
        const double gval = scale * a;
        sum += gval;
        if (odt == HG_DT_F64)
            ((double*)out)[c] = gval - shift;
        else
            ((float*)out)[c] = (float)(gval - shift);
    });
    if (partial) {
        const double v = block_sum(sum, sh);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

__global__ void k_finish_sum(const double* partial, int n, double* out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) v += partial[b];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) *out = v;
}

unsigned blocks_for(const Layout& L) {
    long long rows = (long long)L.ny * L.nz;
    return (unsigned)(rows < kRedBlocks ? rows : kRedBlocks);
}

}  // namespace

int adjoint_inject(hg_grid* a, const void* v, int vdt) {
    hg_grid* g = a;
    k_inject<<<blocks_for(a->L), kThreads, 0, a->stream>>>(a->prec, v, vdt, a->phi[a->cur], a->lo[a->cur],
                                                           a->dlt[a->dcur], a->L);
    HG_LAUNCHED("adjoint injection kernel");
    return HG_OK;
}

int adjoint_accumulate(hg_grid* a, void* acc_a, void* acc_b) {
    hg_grid* g = a;
    k_accumulate<<<blocks_for(a->L), kThreads, 0, a->stream>>>(a->prec, a->phi[a->cur], a->lo[a->cur], acc_a, acc_b,
                                                               a->L);
    HG_LAUNCHED("adjoint accumulation kernel");
    return HG_OK;
}

// dL/drho = -(c dt)^2 4 pi G * acc (dense, into out of type odt on the device), minus its mean when periodic
int adjoint_gradient(hg_grid* a, const void* acc_a, const void* acc_b, void* out, int odt, double* scratch) {
    hg_grid* g = a;
    const double scale = -a->src;
    const unsigned nb = blocks_for(a->L);
    if (a->bc != HG_BC_PERIODIC) {
        k_grad<<<nb, kThreads, 0, a->stream>>>(a->prec, acc_a, acc_b, out, odt, a->L, scale, 0.0, nullptr);
        HG_LAUNCHED("adjoint gradient kernel");
        return HG_OK;
    }
    k_grad<<<nb, kThreads, 0, a->stream>>>(a->prec, acc_a, acc_b, out, odt, a->L, scale, 0.0, scratch);
    HG_LAUNCHED("adjoint gradient kernel");
    k_finish_sum<<<1, kThreads, 0, a->stream>>>(scratch, (int)nb, scratch + kRedBlocks);
    HG_LAUNCHED("adjoint gradient sum kernel");
    double sum = 0.0;
    HG_CUDA(cudaMemcpyAsync(&sum, scratch + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, a->stream));
    HG_CUDA(cudaStreamSynchronize(a->stream));
    const double mean = sum / ((double)a->nx * a->ny * a->nz);
    k_grad<<<nb, kThreads, 0, a->stream>>>(a->prec, acc_a, acc_b, out, odt, a->L, scale, mean, nullptr);
    HG_LAUNCHED("adjoint gradient kernel");
    return HG_OK;
}

}  // namespace hg
