// Two-electron integral columns on the tensor cores (precision form).
//
// X[pq][c] = sum_f m_f conj(phi_p(f)) phi_q(f) Wcol_c(f) over every support
// point f (masters, then hanging points through C): the contraction of the
// n^2 pair densities with the n^2 real mean-field columns that yields the
// integrals (pq|rs) of Eq. ci_eom (Sec. 2; the mean fields of Eq. mean-field,
// Sec. 3.1).  It is a dense product of an (2 n^2 x F) and an (F x n^2) matrix,
// F ~ 10^6 support points, so it runs as tcgen05 MMAs: M = 128 rows (Re and
// Im of the n^2 densities, zero-padded), N = n^2 rounded up to 16, K = 32
// points per tile.  FP32 accuracy from TF32 operands by the split
// x = x_hi + x_lo (three products per tile: hi*hi, hi*lo, lo*hi); each tile's
// FP32 sums are read from tensor memory and added in FP64, one partial row
// set per block, summed by the caller's fixed-order finalize.
//
// One warpgroup per block: all threads stage a tile (densities and columns
// in FP32, converted on the integer pipe), thread 0 issues the tile's MMAs and
// commits them to an mbarrier, and the warps that hold useful accumulator rows
// read them back.  Every wait is bounded; a block that gives up sets *status.
#include "afem_internal.h"
#include "tcgen05.cuh"
#include "vec_common.cuh"

namespace afem {

namespace {

constexpr int kKT = 32;                 // support points per tile (MMA K per tile)
constexpr int kMaxPolls = 1 << 22;      // mbarrier polls before a block gives up

struct TcIntArgs {
    const double2* phi;   // [N][n]
    const double* W;      // [N][nn]
    int n, nn;
    int64_t N, n_int, nh;
    const double* mf_m;
    const double* mf_h;
    const int32_t* hp;
    const int32_t* hm;
    const double* hw;
};

__host__ __device__ constexpr size_t tc_int_smem(int NC) {
    return size_t(2 * 128 + 2 * NC) * kKT * sizeof(float)   // A hi/lo, B hi/lo tiles
           + size_t(kKT) * 8 * sizeof(float2)                 // staged orbitals
           + size_t(kKT) * 64 * sizeof(float)                 // staged W rows
           + size_t(kKT) * sizeof(float);                     // staged m_f
}

template <int NC>
__global__ void __launch_bounds__(128, 1) integrals_tc_kernel(TcIntArgs a, double* __restrict__ partial,
                                                              int* __restrict__ status) {
    constexpr int KT = kKT;
    constexpr uint32_t kCols = NC < 32 ? 32u : uint32_t(NC);   // tensor-memory columns (power of two)
    static_assert(NC == 16 || NC == 32 || NC == 64, "accumulator width");
    constexpr uint32_t kIdesc = tc::idesc_tf32(128, NC);
    constexpr uint32_t kRowStride = (KT / 4) * 128;          // bytes between 8-row groups
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sAh = smem_raw;
    unsigned char* sAl = sAh + 128 * KT * 4;
    unsigned char* sBh = sAl + 128 * KT * 4;
    unsigned char* sBl = sBh + NC * KT * 4;
    float2* s_phi = reinterpret_cast<float2*>(sBl + NC * KT * 4);   // [KT][8]
    float* s_w = reinterpret_cast<float*>(s_phi + KT * 8);           // [KT][64]
    float* s_mf = s_w + KT * 64;                                     // [KT]
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_taddr;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, nn = a.nn;
    // rows beyond 2 nn (A) and nn (B) stay zero for the whole kernel
    for (int i = tid; i < (2 * 128 + 2 * NC) * KT; i += 128) reinterpret_cast<float*>(smem_raw)[i] = 0.f;
    if (tid == 0) tc::mbar_init(&bar, 1);
    if (warp == 0) tc::tmem_alloc(&s_taddr, kCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    const bool holds_rows = warp * 32 < 2 * nn;   // warp-uniform
    double acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.0;
    const int64_t npts = a.N + a.nh;
    const int64_t ntiles = (npts + KT - 1) / KT;
    uint32_t parity = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // 1. stage the tile's orbitals (zero at surface masters), W rows and
        //    m_f in FP32; hanging points interpolated through C in FP64
        const int ncomp = n + nn;
        for (int it = tid; it < KT * ncomp; it += 128) {
            const int t = it / ncomp, j = it - t * ncomp;
            const int64_t f = tile * KT + t;
            if (j < n) {
                double2 v = make_double2(0.0, 0.0);
                if (f < a.N) {
                    if (f < a.n_int) v = a.phi[f * n + j];
                } else if (f < npts) {
                    const int64_t h = f - a.N;
                    for (int e = a.hp[h]; e < a.hp[h + 1]; ++e) {
                        const int64_t m = a.hm[e];
                        if (m < a.n_int) {
                            const double w = a.hw[e];
                            const double2 x = a.phi[m * n + j];
                            v.x = fma(w, x.x, v.x);
                            v.y = fma(w, x.y, v.y);
                        }
                    }
                }
                s_phi[t * 8 + j] = make_float2(narrow_f64(v.x), narrow_f64(v.y));
            } else {
                const int c = j - n;
                double v = 0.0;
                if (f < a.N) {
                    v = a.W[f * nn + c];
                } else if (f < npts) {
                    const int64_t h = f - a.N;
                    for (int e = a.hp[h]; e < a.hp[h + 1]; ++e) v = fma(a.hw[e], a.W[int64_t(a.hm[e]) * nn + c], v);
                }
                s_w[t * 64 + c] = narrow_f64(v);
            }
        }
        for (int t = tid; t < KT; t += 128) {
            const int64_t f = tile * KT + t;
            s_mf[t] = f < a.N ? narrow_f64(a.mf_m[f]) : (f < npts ? narrow_f64(a.mf_h[f - a.N]) : 0.f);
        }
        __syncthreads();
        // 2. operand tiles: A rows 2 pq / 2 pq + 1 = Re / Im of m_f conj(phi_p) phi_q,
        //    B row c = W column c; each value split into TF32 hi and lo.  A warp
        //    writes one 8-row x 4-column core matrix per store (lane = 4 r + k,
        //    128 contiguous bytes: no bank conflicts).
        {
            constexpr int KG = KT / 4;
            const int a_cms = (2 * nn + 7) / 8 * KG;   // core matrices of A holding rows < 2 nn
            const int b_cms = (nn + 7) / 8 * KG;
            for (int cm = warp; cm < a_cms + b_cms; cm += 4) {
                const bool isA = cm < a_cms;
                const int c2 = isA ? cm : cm - a_cms;
                const int row = (c2 / KG) * 8 + (lane >> 2), t = (c2 % KG) * 4 + (lane & 3);
                float v = 0.f;
                if (isA) {
                    if (row < 2 * nn) {
                        const int pq = row >> 1, p = pq / n, q = pq - p * n;
                        const float2 x = s_phi[t * 8 + p], y = s_phi[t * 8 + q];
                        v = s_mf[t] * ((row & 1) ? fmaf(x.x, y.y, -x.y * y.x) : fmaf(x.x, y.x, x.y * y.y));
                    }
                } else if (row < nn) {
                    v = s_w[t * 64 + row];
                }
                const float h = tc::tf32_round(v);
                float* hi = reinterpret_cast<float*>(isA ? sAh : sBh);
                float* lo = reinterpret_cast<float*>(isA ? sAl : sBl);
                hi[c2 * 32 + lane] = h;
                lo[c2 * 32 + lane] = tc::tf32_round(v - h);
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        // 3. the tile's 3 x KT/8 MMAs, issued by one thread
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl);
            const uint32_t bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
#pragma unroll
            for (int s = 0; s < KT / 8; ++s) {
                const uint32_t off = uint32_t(s) * 256u;
                const uint64_t dah = tc::smem_desc(ah + off, 128, kRowStride);
                const uint64_t dal = tc::smem_desc(al + off, 128, kRowStride);
                const uint64_t dbh = tc::smem_desc(bh + off, 128, kRowStride);
                const uint64_t dbl = tc::smem_desc(bl + off, 128, kRowStride);
                tc::mma_tf32(taddr, dal, dbh, kIdesc, s > 0);
                tc::mma_tf32(taddr, dah, dbl, kIdesc, true);
                tc::mma_tf32(taddr, dah, dbh, kIdesc, true);
            }
            tc::commit(&bar);
        }
        // 4. wait for the MMAs (bounded), then add the tile's FP32 sums in FP64
        const bool got = tc::mbar_wait(&bar, parity, kMaxPolls);
        parity ^= 1u;
        if (__syncthreads_or(!got)) {
            ok = false;
            break;
        }
        tc::fence_after_sync();
        if (holds_rows) {
#pragma unroll
            for (int c0 = 0; c0 < NC; c0 += 16) {
                float v[16];
                tc::ld_x16(taddr + (uint32_t(warp * 32) << 16) + uint32_t(c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[c0 + j] += widen_f32(v[j]);
            }
        }
        tc::fence_before_sync();
        __syncthreads();   // tiles and accumulator free for the next tile
    }
    const int row = warp * 32 + lane;
    if (ok) {
        if (row < 2 * nn) {
            const int pq = row >> 1, part = row & 1;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (c < nn) partial[((int64_t(blockIdx.x) * nn + pq) * nn + c) * 2 + part] = acc[c];
        }
    } else {
        if (tid == 0) atomicExch(status, 1);
        // the MMAs of the abandoned tile may still run: wait for them once more
        // (bounded) before the columns are freed
        tc::mbar_wait(&bar, parity ^ 1u, kMaxPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(taddr, kCols);
}

template <int NC>
int launch_tc(const TcIntArgs& a, double2* partial, int grid, int* status, cudaStream_t s) {
    const size_t smem = tc_int_smem(NC);
    AFEM_CUDA_TRY(allow_dyn_smem(integrals_tc_kernel<NC>));
    AFEM_LAUNCH((integrals_tc_kernel<NC>), grid, 128, smem, s, a, reinterpret_cast<double*>(partial), status);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

}  // namespace

int integrals_tc(const afem_mesh* m, const double2* phi, const double* W, int n, double2* partial, int grid,
                 int* status, cudaStream_t s) {
    if (n < 1 || n > 8) return set_error(AFEM_EINVAL, "integrals_tc: orbital count must be 1..8");
    const DeviceMesh& D = m->dev;
    const int nn = n * n;
    TcIntArgs a{phi, W, n, nn, D.n_master, D.n_interior, D.n_hanging, D.mf_master, D.mf_hang,
                D.hang_ptr, D.hang_master, D.hang_w};
    if (nn <= 16) return launch_tc<16>(a, partial, grid, status, s);
    if (nn <= 32) return launch_tc<32>(a, partial, grid, status, s);
    return launch_tc<64>(a, partial, grid, status, s);
}

}  // namespace afem
