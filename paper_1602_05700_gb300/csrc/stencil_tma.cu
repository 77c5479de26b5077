// TMA-staged single sweep of the compensated-float sub-step (arXiv 1602.05700, Sec. 1 Eq. HNeq., Sec. 2): the
// kernel of a single grid's sub-step (the sweep itself is tma_sweep in sweep_tma.cuh), and the host side of the
// staging -- the 3-D tensor maps of a grid's state, built once through the driver's cuTensorMapEncodeTiled, and the
// entries of the batched launch.
#include <cuda.h>

#include "sweep_tma.cuh"

namespace hg {

namespace {

template <int WY, int S>
__global__ void __launch_bounds__(32 * (WY + 1), 3)
    k_step_f32k_tma(const __grid_constant__ CUtensorMap m_hi, const __grid_constant__ CUtensorMap m_lo,
                    const __grid_constant__ CUtensorMap m_d, const __grid_constant__ CUtensorMap m_s,
                    const SweepArgs A, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[2 * S];
    tma_sweep<WY, S>(&m_hi, &m_lo, &m_d, &m_s, A, blockIdx.x, blockIdx.y, blockIdx.z, err, smem, bars);
}

// the bounded-wait path itself: an mbarrier that nothing ever arrives on, waited for with a short limit
__global__ void k_wait_selftest(int* err, unsigned long long limit_ns) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    mbar_wait(smem_addr(&bar), 0u, err, limit_ns);
}

// the index check itself: the index one past the padded array goes to the same check the sub-step kernels use;
// nothing is stored, whatever the check answers
__global__ void k_bounds_selftest(long long elems, int* err) { (void)idx_ok(elems, 1, elems, err); }

using TmaEncode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_fn(TmaEncode* fn) {
    static TmaEncode cached = nullptr;
    if (!cached) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return fail(HG_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        cached = (TmaEncode)p;
    }
    *fn = cached;
    return HG_OK;
}

}  // namespace

// a 3-D map over a padded array (pitch x (ny+2) x (nz+2) elements of `bytes` each) with boxes of box_x x box_y x 1
int tma_encode(CUtensorMap* m, void* base, const Layout& L, int bytes, int box_x, int box_y) {
    TmaEncode fn;
    int rc = encode_fn(&fn);
    if (rc) return rc;
    const cuuint64_t dim[3] = {(cuuint64_t)L.pitch, (cuuint64_t)(L.ny + 2), (cuuint64_t)(L.nz + 2)};
    const cuuint64_t stride[2] = {(cuuint64_t)L.pitch * bytes, (cuuint64_t)L.plane * bytes};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    const cuuint32_t estride[3] = {1, 1, 1};
    CUresult r = fn(m, bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, base, dim,
                    stride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(HG_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return HG_OK;
}

// tensor maps of the compensated-float state: hi[0..1], lo[0..1], dlt[0..1] (dlt[1] once it exists), s
int tma_maps(hg_grid* g) {
    if (g->tm_ready == (g->dlt[1] ? 2 : 1)) return HG_OK;
    const Layout& L = g->L;
    int rc;
    for (int b = 0; b < 2; ++b) {
        if ((rc = tma_encode(&g->tm[0 + b], g->phi[b], L, 4, kHX, kTmaWY + 2))) return rc;
        if ((rc = tma_encode(&g->tm[2 + b], g->lo[b], L, 2, kHX, kTmaWY + 2))) return rc;
        if (g->dlt[b] && (rc = tma_encode(&g->tm[4 + b], g->dlt[b], L, 4, kTX, kTmaWY))) return rc;
    }
    if ((rc = tma_encode(&g->tm[6], g->rho, L, 4, kTX, kTmaWY))) return rc;
    g->tm_ready = g->dlt[1] ? 2 : 1;
    return HG_OK;
}

static constexpr int kSmem = kStages * StageGeom<kTmaWY>::bytes;

// the interior sweep of one compensated-float sub-step (cur -> 1 - cur), staged through shared memory by TMA
int launch_sweep_f32k_tma(hg_grid* g, const SweepArgs& A) {
    int rc = tma_maps(g);
    if (rc) return rc;
    static unsigned long long attr_done = 0;
    const int smem = kSmem;
    if ((rc = smem_attr_once((const void*)k_step_f32k_tma<kTmaWY, kStages>, smem, &attr_done))) return rc;
    const int c = g->cur;
    dim3 grid((g->nx + kTX - 1) / kTX, (g->ny + kTmaWY - 1) / kTmaWY, (g->nz + A.zb - 1) / A.zb);
    SweepArgs At = A;
    At.gx = grid.x;
    At.gy = grid.y;
    k_step_f32k_tma<kTmaWY, kStages><<<grid, 32 * (kTmaWY + 1), smem, g->stream>>>(
        g->tm[0 + c], g->tm[2 + c], g->tm[4 + g->dcur], g->tm[6], At, g->derr);
    HG_LAUNCHED("TMA-staged sub-step kernel");
    return HG_OK;
}

// the batched-launch entry of grid g for its sub-step cur -> 1 - cur: Robin ghosts of all faces inside the launch,
// periodic ghosts by the blocks' epilogue
int tma_entry(hg_grid* g, TmaEntry* e, int zb) {
    int rc = tma_maps(g);
    if (rc) return rc;
    const int c = g->cur;
    e->m[0] = g->tm[0 + c];
    e->m[1] = g->tm[2 + c];
    e->m[2] = g->tm[4 + g->dcur];
    e->m[3] = g->tm[6];
    e->A = sweep_args(g, zb);
    e->A.gx = (g->nx + kTX - 1) / kTX;
    e->A.gy = (g->ny + kTmaWY - 1) / kTmaWY;
    e->A.B.xfaces = 0;
    e->err = g->derr;
    return HG_OK;
}

int bounds_selftest(hg_grid* g) {
    k_bounds_selftest<<<1, 1, 0, g->stream>>>(g->L.elems, g->derr);
    HG_LAUNCHED("index-check self-test kernel");
    return HG_OK;
}

int wait_selftest(hg_grid* g) {
    k_wait_selftest<<<1, 32, 0, g->stream>>>(g->derr, 1000000ull);  // 1 ms
    HG_LAUNCHED("bounded-wait self-test kernel");
    return device_error(g);
}

}  // namespace hg
