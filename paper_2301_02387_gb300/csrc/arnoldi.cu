// Short-iterative Arnoldi propagation of all orbitals at once (Sec. 3.2).
//
// With phi, the RDMs, the mean fields and the field frozen at t, the packed
// orbital equation (Eq. packed_orb_eom) is linear, i d(phi)/dt = G phi, and
// phi(t + dt) = exp(-i G dt) phi(t).  The Krylov space of G from phi is built
// by Arnoldi in the inner product <u, v> = sum_p u_p^H M_L v_p; then
// phi(t+dt) = beta V_m exp(-i dt H_m) e_1.
// G applied to the stacked orbitals v (Eqs. orb_eom / discretized_eom, X = 0):
//   z_p = H1~ v_p + C^T diag(m_f) sum_q (C U_pq) o (C v_q)      (one cell pass)
//   y_p = M_L^-1 z_p,   (G v)_p = y_p - sum_j phi_j (phi_j^H M_L y_p)
// and phi_j^H M_L y_p = phi_j^H z_p, so the projector needs no extra scaling.
//
// Orthogonalisation: classical Gram-Schmidt, one pass for all inner products
// (fused with the projector pass of G) and one for the update, plus a second
// pair of passes only when the update cancelled the vector to below 1e-2 of
// its norm (the Daniel-Gragg-Kaufman-Stewart test with a loose threshold).
// GB300 runs FP64 at about 1/64 of its FP32 rate, so these vector kernels
// are bound by FP64 instructions rather than by HBM: each keeps the FP64
// work per element at 4 multiply-adds per basis vector and pass, and in the
// precision form the projector (part of applying G) runs in FP32.  The
// Hessenberg matrix and the norms stay on the device; the host waits once
// per substep, after the candidate substep exponentials are evaluated.
#include <algorithm>
#include <cmath>
#include <vector>

#include "afem_internal.h"
#include "arnoldi.cuh"
#include "vec_common.cuh"

namespace afem {

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }

// S[a][b] = sum_k w_k conj(A[k][a]) B[k][b] over rows k < n_rows (w_k = 1 when
// w is null), reduced in the same launch: partial rows of 2*kout doubles (re,
// im interleaved); the last block writes out[kout].  diag != 0: only a == b
// (kout = na), else all na*nb pairs (kout = na*nb <= 256).
template <typename TB>
__global__ void cdot_fused_kernel(const double2* __restrict__ A, int na, const TB* __restrict__ B, int nb,
                                  const double* __restrict__ w, int64_t n_rows, int diag, double* __restrict__ partial,
                                  unsigned* __restrict__ counter, double2* __restrict__ out) {
    __shared__ double sx[kRedThreads], sy[kRedThreads];
    const int kout = diag ? na : na * nb;
    const int R = kRedThreads / kout, used = R * kout;
    const int t = threadIdx.x;
    double ax = 0.0, ay = 0.0;
    if (t < used) {
        const int o = t % kout, r = t / kout;
        const int ia = diag ? o : o / nb;
        const int ib = diag ? o : o - ia * nb;
        for (int64_t k = int64_t(blockIdx.x) * R + r; k < n_rows; k += int64_t(gridDim.x) * R) {
            double2 u = A[k * na + ia];
            const double2 v = to_d2(B[k * nb + ib]);
            if (w) {
                const double wk = w[k];
                u = make_double2(wk * u.x, wk * u.y);
            }
            ax = fma(u.x, v.x, fma(u.y, v.y, ax));
            ay = fma(u.x, v.y, fma(-u.y, v.x, ay));
        }
    }
    sx[t] = ax;
    sy[t] = ay;
    __syncthreads();
    for (int o = t; o < kout; o += blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int r = 0; r < R; ++r) {
            x += sx[o + kout * r];
            y += sy[o + kout * r];
        }
        partial[int64_t(blockIdx.x) * 2 * kout + 2 * o] = x;
        partial[int64_t(blockIdx.x) * 2 * kout + 2 * o + 1] = y;
    }
    if (!last_block_sum(partial, 2 * kout, counter, sx)) return;
    for (int o = t; o < kout; o += blockDim.x) out[o] = make_double2(sx[2 * o], sx[2 * o + 1]);
}

// Thread layout of the row-major [rows][n] vector kernels: thread t < n*R of a
// 256-thread block owns column p = t % n of rows r = t / n, r + R, ... within
// the block's row range (R = 256 / n), so consecutive threads touch
// consecutive elements and no element index is divided.
struct RowCol {
    int p, r, R;
    bool active;
    __device__ __forceinline__ RowCol(int n) {
        R = kRedThreads / n;
        active = int(threadIdx.x) < n * R;
        r = active ? int(threadIdx.x) / n : 0;
        p = active ? int(threadIdx.x) - r * n : 0;
    }
};

// Sums of v[0..cnt) over the block; the block's row partial[blockIdx][0..cnt)
// is written.  FP64 adds are the scarce resource on GB300, so for more than
// a few values the sums go through shared memory in chunks of 8 values
// (transposed: warp j sums value j of the chunk, 8 adds per lane and a 5-step
// shuffle) instead of a 5-step shuffle per value and thread: about 1.6 FP64
// adds per value and thread instead of 5.
template <int MAXV>
__device__ __forceinline__ void block_row_partial(double (&v)[MAXV], int cnt, double* __restrict__ partial) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (MAXV < 4) {
        __shared__ double s_w[kRedThreads / 32][MAXV];
#pragma unroll
        for (int i = 0; i < MAXV; ++i) {
            if (i < cnt) {
                double x = v[i];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
                if (lane == 0) s_w[warp][i] = x;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            double x = 0.0;
            for (int w = 0; w < kRedThreads / 32; ++w) x += s_w[w][i];
            partial[int64_t(blockIdx.x) * cnt + i] = x;
        }
    } else {
        static_assert(kRedThreads == 256, "the chunked block sum assumes 8 warps of 32");
        __shared__ double s_t[8][kRedThreads + 8];
        const int t = threadIdx.x;
#pragma unroll
        for (int c0 = 0; c0 < MAXV; c0 += 8) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (c0 + j < MAXV) s_t[j][t + (t >> 5)] = v[c0 + j];   // padded against bank conflicts
            __syncthreads();
            if (c0 + warp < cnt) {
                double x = 0.0;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int src = lane * 8 + r;
                    x += s_t[warp][src + (src >> 5)];
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
                if (lane == 0) partial[int64_t(blockIdx.x) * cnt + c0 + warp] = x;
            }
            __syncthreads();
        }
    }
}

// Projector overlaps of the precision form, S[a][b] = sum_k conj(A[k][a]) B[k][b]
// over interior rows from complex64 inputs (NO = n orbitals), added in FP64 into
// slot (block % kOvSlots) of slots[kOvSlots][2 NO^2] (re, im interleaved; the
// consumer sums the slots and clears them).  For even NO two threads share a
// row, each forming the products of half the rows a of S in FP32 registers
// (fewer registers, more rows in flight); the block sums its threads' values in
// FP32 over 8 segments of 32 threads (through shared memory, transposed) and
// the segment sums in FP64.  S is consumed in FP32 by the projector, and the
// FP64 work is per block, with no last-block pass.
constexpr int kOvSlots = 16;
template <int NO>
__global__ void __launch_bounds__(kRedThreads) overlap32_kernel(const float2* __restrict__ A,
                                                                const float2* __restrict__ B, int64_t n_rows,
                                                                double* __restrict__ slots) {
    constexpr int HS = NO % 2 == 0 ? 2 : 1;   // threads per row
    constexpr int NA = NO / HS;               // rows a of S per thread
    constexpr int CNT = 2 * NO * NO;          // values of S
    constexpr int CT = 2 * NA * NO;           // values per thread
    const int t = threadIdx.x;
    const int h = HS == 2 ? (t & 1) : 0;
    float f[CT];
#pragma unroll
    for (int i = 0; i < CT; ++i) f[i] = 0.f;
    const int rows_per_block = kRedThreads / HS;
#pragma unroll 2
    for (int64_t k = blockIdx.x * int64_t(rows_per_block) + t / HS; k < n_rows;
         k += int64_t(gridDim.x) * rows_per_block) {
        float2 a[NA], b[NO];
#pragma unroll
        for (int i = 0; i < NA; ++i) a[i] = A[k * NO + h * NA + i];
        if constexpr (NO % 2 == 0) {   // a row of B is NO/2 16-byte words
            const float4* B4 = reinterpret_cast<const float4*>(B + k * NO);
#pragma unroll
            for (int i = 0; i < NO / 2; ++i) {
                const float4 ub = B4[i];
                b[2 * i] = make_float2(ub.x, ub.y);
                b[2 * i + 1] = make_float2(ub.z, ub.w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NO; ++i) b[i] = B[k * NO + i];
        }
#pragma unroll
        for (int i = 0; i < NA; ++i)
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                f[2 * (i * NO + j)] = fmaf(a[i].x, b[j].x, fmaf(a[i].y, b[j].y, f[2 * (i * NO + j)]));
                f[2 * (i * NO + j) + 1] = fmaf(a[i].x, b[j].y, fmaf(-a[i].y, b[j].x, f[2 * (i * NO + j) + 1]));
            }
    }
    static_assert(kRedThreads == 256, "the segment sums assume 8 warps of 32");
    __shared__ float s_t[32][kRedThreads + 1];   // a chunk of 32 values x 256 threads
    __shared__ float s_seg[8][32];
    const int lane = t & 31, seg = t >> 5;
    double* slot = slots + int64_t(blockIdx.x % kOvSlots) * CNT;
#pragma unroll
    for (int c0 = 0; c0 < CNT; c0 += 32) {
        // value c0 + j of S is this thread's f[c0 + j - h CT] when that index is its own
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (c0 + j < CNT) {
                float v = 0.f;
                if (h == 0) {
                    if (c0 + j < CT) v = f[c0 + j < CT ? c0 + j : 0];
                } else {
                    if (c0 + j >= CT) v = f[c0 + j >= CT ? c0 + j - CT : 0];
                }
                s_t[j][t] = v;
            }
        }
        __syncthreads();
        if (c0 + lane < CNT) {   // value c0 + lane over the 32 threads of segment seg
            float x = 0.f;
#pragma unroll 8
            for (int r = 0; r < 32; ++r) x += s_t[lane][seg * 32 + r];
            s_seg[seg][lane] = x;
        }
        __syncthreads();
        if (t < 32 && c0 + t < CNT) {
            double x = 0.0;
#pragma unroll
            for (int g = 0; g < 8; ++g) x += widen_f32(s_seg[g][t]);
            atomicAdd(slot + c0 + t, x);
        }
        __syncthreads();
    }
}

// acc[2i], acc[2i+1] += conj(u_i) mx (i < NV) and acc[2NV] += conj(x) mx, with
// mx = m x formed once: 4 FP64 multiply-adds per basis vector.
template <int NV>
__device__ __forceinline__ void accumulate_dots(double (&acc)[2 * NV + 1], const double2 (&u)[NV > 0 ? NV : 1],
                                                double2 x, double m) {
    const double2 mx = make_double2(m * x.x, m * x.y);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        acc[2 * i] = fma(u[i].x, mx.x, fma(u[i].y, mx.y, acc[2 * i]));
        acc[2 * i + 1] = fma(u[i].x, mx.y, fma(-u[i].y, mx.x, acc[2 * i + 1]));
    }
    // the norm only without basis vectors; with them finish_dots takes the
    // in-span part of the norm from the inner products (no FP64 work per element)
    if constexpr (NV == 0) acc[0] = fma(x.x, mx.x, fma(x.y, mx.y, acc[0]));
}

// Krylov vectors are stored unscaled: V_0 is the substep's start vector and
// V_{i+1} the raw Gram-Schmidt remainder of the cell pass applied to V_i, with
// q_i = s_f[i] V_i, s_f[0] = 1 / beta, s_f[i] = s_f[i-1] / h_{i,i-1} (= 1 / |V_i|_M),
// so no pass over the basis only to scale it and no FP64 scaling of the new
// vector (0 after a breakdown, h <= 1e-14 beta).  Callers __syncthreads()
// before use.
__device__ __forceinline__ void krylov_scales(const double2* __restrict__ H, int ldh,
                                              const double2* __restrict__ beta2, int nv, double* s_f) {
    if (threadIdx.x != 0 || nv <= 0) return;
    const double beta = sqrt(fmax(beta2->x, 0.0));
    double f = beta > 0.0 ? 1.0 / beta : 0.0;
    s_f[0] = f;
    for (int i = 1; i < nv; ++i) {
        const double h = H[(i - 1) * ldh + i].x;
        f = (h > 1e-14 * beta && h > 0.0) ? f / h : 0.0;
        s_f[i] = f;
    }
}

// The block sums of acc (inner products of the raw vector w with the stored
// V_i), then in the last block the true values for the vector fw w with
// fw = s_f[NV-1] (1 when NV = 0): out[i] = s_f[i] fw (acc[2i], acc[2i+1]) =
// <q_i, fw w> for i < NV and out[NV] = (sum_i |out[i]|^2, 0), the squared
// norm of the part of fw w in the span of q_0..q_{NV-1} (for NV = 0,
// |w|^2 itself).  By Pythagoras the norm before the update is this plus the
// norm the update leaves, which is how the re-orthogonalisation test uses it.
template <int NV>
// Returns true in the last block (after every block has finished its reads).
__device__ __forceinline__ bool finish_dots(double (&acc)[2 * NV + 1], const double* s_f,
                                            double* __restrict__ partial, unsigned* __restrict__ counter,
                                            double2* __restrict__ out) {
    constexpr int CNT = NV > 0 ? 2 * NV : 1;
    block_row_partial<2 * NV + 1>(acc, CNT, partial);
    __shared__ double s_sum[kRedThreads];
    if (!last_block_sum(partial, CNT, counter, s_sum)) return false;
    const double fw = NV > 0 ? s_f[NV > 0 ? NV - 1 : 0] : 1.0;
    for (int i = threadIdx.x; i < NV; i += blockDim.x) {
        const double f = s_f[i] * fw;
        out[i] = make_double2(f * s_sum[2 * i], f * s_sum[2 * i + 1]);
    }
    if (threadIdx.x == 0) {
        double nn = 0.0;
        if (NV == 0) {
            nn = s_sum[0];
        } else {
            for (int i = 0; i < NV; ++i) {
                const double f = s_f[i] * fw;
                nn += f * f * (s_sum[2 * i] * s_sum[2 * i] + s_sum[2 * i + 1] * s_sum[2 * i + 1]);
            }
        }
        out[NV] = make_double2(nn, 0.0);
    }
    return true;
}

// Gram-Schmidt inner products: out[i] = <q_i, w>_M for i < NV and out[NV] as
// finish_dots states, over interior rows.  Skipped when gate && !*gate.
// NV is a template parameter so that the NV + 1 loads of a row are issued
// back to back before any of them is used.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) krylov_dots_kernel(
    const double2* __restrict__ w, const double2* __restrict__ V, int64_t stride, const double* __restrict__ ml,
    int64_t n_int, int n, const int* __restrict__ gate, const double2* __restrict__ H, int ldh,
    const double2* __restrict__ beta2, double* __restrict__ partial, unsigned* __restrict__ counter,
    double2* __restrict__ out) {
    if (gate && *gate == 0) return;
    __shared__ double s_f[NV > 0 ? NV : 1];
    if (NV > 0) krylov_scales(H, ldh, beta2, NV, s_f);
    double acc[2 * NV + 1];
#pragma unroll
    for (int i = 0; i < 2 * NV + 1; ++i) acc[i] = 0.0;
    const RowCol rc(n);
    if (rc.active) {
        for (int64_t k = int64_t(blockIdx.x) * rc.R + rc.r; k < n_int; k += int64_t(gridDim.x) * rc.R) {
            const int64_t o = k * n + rc.p;
            const double m = ml[k];
            const double2 x = w[o];
            double2 u[NV > 0 ? NV : 1];
#pragma unroll
            for (int i = 0; i < NV; ++i) u[i] = V[i * stride + o];
            accumulate_dots<NV>(acc, u, x, m);
        }
    }
    finish_dots<NV>(acc, s_f, partial, counter, out);
}

// The projector pass of G fused with the first Gram-Schmidt pass (FP64 form):
// z is the cell pass applied to the stored V_{NV-1}, so the raw vector
// w[k][p] = ML^-1[k] z[k][p] - sum_j phi[k][j] S[j][p] on interior rows (0 on
// the others) is G q_{NV-1} / s_f[NV-1]; it is written unscaled, and
// out[i] = <q_i, G q_{NV-1}>_M (i < NV) and out[NV] (see finish_dots) are
// formed from the values in registers, so w is not read back.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) project_dots_kernel(
    const double2* __restrict__ z, const double2* __restrict__ phi, const double2* __restrict__ S,
    const double* __restrict__ ml_inv, const double* __restrict__ ml, int64_t n_int, int64_t N, int n,
    double2* __restrict__ w, const double2* __restrict__ V, int64_t stride, const double2* __restrict__ H, int ldh,
    const double2* __restrict__ beta2, double* __restrict__ partial, unsigned* __restrict__ counter,
    double2* __restrict__ out) {
    __shared__ double2 s_S[kMaxOrbProj * kMaxOrbProj];
    __shared__ double s_f[NV];
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) s_S[i] = S[i];
    krylov_scales(H, ldh, beta2, NV, s_f);
    __syncthreads();
    double acc[2 * NV + 1];
#pragma unroll
    for (int i = 0; i < 2 * NV + 1; ++i) acc[i] = 0.0;
    const RowCol rc(n);
    if (rc.active) {
        const int p = rc.p;
        for (int64_t k = int64_t(blockIdx.x) * rc.R + rc.r; k < N; k += int64_t(gridDim.x) * rc.R) {
            const int64_t o = k * n + p;
            double2 x = make_double2(0.0, 0.0);
            if (k < n_int) {
                double2 u[NV];
#pragma unroll
                for (int i = 0; i < NV; ++i) u[i] = V[i * stride + o];
                const double s = ml_inv[k];
                const double2 zo = z[o];
                x = make_double2(zo.x * s, zo.y * s);
                for (int j = 0; j < n; ++j) {
                    const double2 f = phi[k * n + j];
                    const double2 c = s_S[j * n + p];
                    x.x = fma(-f.x, c.x, fma(f.y, c.y, x.x));
                    x.y = fma(-f.x, c.y, fma(-f.y, c.x, x.y));
                }
                accumulate_dots<NV>(acc, u, x, ml[k]);
            }
            w[o] = x;
        }
    }
    finish_dots<NV>(acc, s_f, partial, counter, out);
}

// The same for the precision form: the projector in FP32 from the complex64
// cell-pass output z and the complex64 orbitals phi32 (part of applying G),
// the result widened to FP64 for the Gram-Schmidt inner products.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) project32_dots_kernel(
    const float2* __restrict__ z, const float2* __restrict__ phi, const double2* __restrict__ S,
    const float* __restrict__ ml_inv, const double* __restrict__ ml, int64_t n_int, int64_t N, int n,
    double2* __restrict__ w, const double2* __restrict__ V, int64_t stride, const double2* __restrict__ H, int ldh,
    const double2* __restrict__ beta2, double* __restrict__ partial, unsigned* __restrict__ counter,
    double2* __restrict__ out, double* __restrict__ S_slots) {
    __shared__ float2 s_S[kMaxOrbProj * kMaxOrbProj];
    __shared__ double s_f[NV];
    // the overlaps: the sum of overlap32_kernel's slots (cleared by the last
    // block below), or S itself (zero without the projector)
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        if (S_slots) {
            double x = 0.0, y = 0.0;
            for (int sl = 0; sl < kOvSlots; ++sl) {
                x += S_slots[sl * 2 * n * n + 2 * i];
                y += S_slots[sl * 2 * n * n + 2 * i + 1];
            }
            s_S[i] = make_float2(narrow_f64(x), narrow_f64(y));
        } else {
            s_S[i] = make_float2(narrow_f64(S[i].x), narrow_f64(S[i].y));
        }
    }
    krylov_scales(H, ldh, beta2, NV, s_f);
    __syncthreads();
    // the complex64 input of the cell pass was 2^kv V_{NV-1} (krylov_update_kernel's
    // scaling; V_0 unscaled), so the raw vector is the result times 2^-kv
    const int kv = (NV >= 2 && s_f[NV >= 2 ? NV - 2 : 0] > 0.0) ? ilogb(s_f[NV >= 2 ? NV - 2 : 0]) : 0;
    double acc[2 * NV + 1];
#pragma unroll
    for (int i = 0; i < 2 * NV + 1; ++i) acc[i] = 0.0;
    const RowCol rc(n);
    if (rc.active) {
        const int p = rc.p;
        for (int64_t k = int64_t(blockIdx.x) * rc.R + rc.r; k < N; k += int64_t(gridDim.x) * rc.R) {
            const int64_t o = k * n + p;
            double2 x = make_double2(0.0, 0.0);
            if (k < n_int) {
                double2 u[NV];
#pragma unroll
                for (int i = 0; i < NV; ++i) u[i] = V[i * stride + o];
                const float s = ml_inv[k];
                const float2 zo = z[o];
                float2 xf = make_float2(zo.x * s, zo.y * s);
                for (int j = 0; j < n; ++j) {
                    const float2 f = phi[k * n + j];
                    const float2 c = s_S[j * n + p];
                    xf.x = fmaf(-f.x, c.x, fmaf(f.y, c.y, xf.x));
                    xf.y = fmaf(-f.x, c.y, fmaf(-f.y, c.x, xf.y));
                }
                x = make_double2(widen_f32_scaled(xf.x, -kv), widen_f32_scaled(xf.y, -kv));
                accumulate_dots<NV>(acc, u, x, ml[k]);
            }
            w[o] = x;
        }
    }
    if (finish_dots<NV>(acc, s_f, partial, counter, out) && S_slots)
        for (int o = threadIdx.x; o < kOvSlots * 2 * n * n; o += blockDim.x) S_slots[o] = 0.0;
}

// Gram-Schmidt update of the raw vector w (the true vector is fw w with
// fw = s_f[NV-1]): fw w -= sum_{i<NV} c_i q_i, i.e. w -= sum_i (c_i s_f[i] / fw)
// V_i (interior rows), with the new norm, and the complex64 copy of w in w32
// when non-null (the input of the next cell pass); the last block writes the
// Hessenberg column: Hcol[i] = c_i (or += c_i when accumulate),
// Hcol[NV] = fw |w|_M, and *reorth = 1 when a first pass left
// |fw w|^2 < eta2 (c[NV] + |fw w|^2), the squared norm before it (c[NV] is
// its part in the span of the basis).  Skipped when gate && !*gate.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) krylov_update_kernel(
    double2* __restrict__ w, const double2* __restrict__ V, int64_t stride, const double2* __restrict__ c,
    const double* __restrict__ ml, int64_t n_int, int n, const int* __restrict__ gate, int accumulate, double eta2,
    int* __restrict__ reorth, const double2* __restrict__ H, int ldh, const double2* __restrict__ beta2,
    float2* __restrict__ w32, double* __restrict__ partial, unsigned* __restrict__ counter,
    double2* __restrict__ Hcol) {
    if (gate && *gate == 0) return;
    __shared__ double2 s_c[NV + 1];
    __shared__ double2 s_cf[NV];
    __shared__ double s_f[NV];
    krylov_scales(H, ldh, beta2, NV, s_f);
    if (int(threadIdx.x) <= NV) s_c[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    const double fw = s_f[NV - 1];
    // the complex64 copy holds 2^kw w with 2^kw ~ fw, i.e. about the true vector
    // fw w (whose size is the Hessenberg entry): the raw vectors grow like the
    // operator norm to the power of their index and would leave the binary32
    // range (project32_dots_kernel undoes the factor)
    const int kw = fw > 0.0 ? ilogb(fw) : 0;
    if (int(threadIdx.x) < NV) {
        const double f = fw > 0.0 ? s_f[threadIdx.x] / fw : 0.0;
        s_cf[threadIdx.x] = make_double2(s_c[threadIdx.x].x * f, s_c[threadIdx.x].y * f);
    }
    __syncthreads();
    double nrm[1] = {0.0};
    const RowCol rc(n);
    if (rc.active) {
        for (int64_t k = int64_t(blockIdx.x) * rc.R + rc.r; k < n_int; k += int64_t(gridDim.x) * rc.R) {
            const int64_t o = k * n + rc.p;
            double2 x = w[o];
            const double m = ml[k];
            double2 u[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) u[i] = V[i * stride + o];
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const double2 h = s_cf[i];
                x.x = fma(-h.x, u[i].x, fma(h.y, u[i].y, x.x));
                x.y = fma(-h.x, u[i].y, fma(-h.y, u[i].x, x.y));
            }
            w[o] = x;
            if (w32) w32[o] = make_float2(narrow_f64_scaled(x.x, kw), narrow_f64_scaled(x.y, kw));
            nrm[0] = fma(m, fma(x.x, x.x, x.y * x.y), nrm[0]);
        }
    }
    block_row_partial<1>(nrm, 1, partial);
    __shared__ double s_sum[kRedThreads];
    if (!last_block_sum(partial, 1, counter, s_sum)) return;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NV; ++i) {
            const double2 hh = accumulate ? make_double2(Hcol[i].x + s_c[i].x, Hcol[i].y + s_c[i].y) : s_c[i];
            Hcol[i] = hh;
        }
        const double nn = fw * fw * fmax(s_sum[0], 0.0);   // |fw w|^2
        Hcol[NV] = make_double2(sqrt(nn), 0.0);
        // |fw w|^2 before the update = in-span part (c[NV]) + what is left (nn)
        if (reorth) *reorth = (!accumulate && nn < eta2 * (s_c[NV].x + nn)) ? 1 : 0;
    }
}

// Closes a substep and opens the next: x = scale sum_{i<M} y_i q_i (q_i =
// s_f[i] V_i) is written to out (phi after the substep) and, as the next
// substep's unscaled V_0, to V itself (element by element after its reads),
// with the complex64 copy in v32 when non-null; the last block writes
// beta2_out = |x|_M^2 over interior rows.  M = 0 opens the first substep
// from src (out unused).  beta2_out may be beta2: every block reads beta2 at
// its start and the last block writes after all others have finished.
template <int M>
__global__ void __launch_bounds__(kRedThreads) substep_close_kernel(
    double2* V, int64_t stride, const double2* __restrict__ y, double scale, const double2* __restrict__ H, int ldh,
    const double2* beta2, const double2* __restrict__ src, const double* __restrict__ ml, int64_t n_int, int64_t N,
    int n, double2* __restrict__ out, float2* __restrict__ v32, double* __restrict__ partial,
    unsigned* __restrict__ counter, double2* beta2_out) {
    __shared__ double2 s_y[M > 0 ? M : 1];
    __shared__ double s_f[M > 0 ? M : 1];
    if (M > 0) krylov_scales(H, ldh, beta2, M, s_f);
    __syncthreads();
    if (int(threadIdx.x) < M) {
        const double f = scale * s_f[threadIdx.x];
        s_y[threadIdx.x] = make_double2(f * y[threadIdx.x].x, f * y[threadIdx.x].y);
    }
    __syncthreads();
    double nrm[1] = {0.0};
    const RowCol rc(n);
    if (rc.active) {
        for (int64_t k = int64_t(blockIdx.x) * rc.R + rc.r; k < N; k += int64_t(gridDim.x) * rc.R) {
            const int64_t o = k * n + rc.p;
            double2 x;
            if (M == 0) {
                x = src[o];
            } else {
                double2 u[M > 0 ? M : 1];
#pragma unroll
                for (int i = 0; i < M; ++i) u[i] = V[i * stride + o];
                x = make_double2(0.0, 0.0);
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const double2 c = s_y[i];
                    x.x = fma(c.x, u[i].x, fma(-c.y, u[i].y, x.x));
                    x.y = fma(c.x, u[i].y, fma(c.y, u[i].x, x.y));
                }
                out[o] = x;
            }
            V[o] = x;
            if (v32) v32[o] = make_float2(narrow_f64(x.x), narrow_f64(x.y));
            if (k < n_int) nrm[0] = fma(ml[k], fma(x.x, x.x, x.y * x.y), nrm[0]);
        }
    }
    block_row_partial<1>(nrm, 1, partial);
    __shared__ double s_sum[kRedThreads];
    if (!last_block_sum(partial, 1, counter, s_sum)) return;
    if (threadIdx.x == 0) *beta2_out = make_double2(fmax(s_sum[0], 0.0), 0.0);
}

// exp(-i dt H) (imag: exp(-dt H), the imaginary-time step) for an m x m
// complex matrix (m <= kMaxKrylov) by one block: scaling and squaring with a
// truncated Taylor series (the scaled matrix has 1-norm <= 1/2; the remainder
// after 16 terms is below 0.5^17 / 17! ~ 2e-20 relative, under the FP64
// rounding of the squarings).
constexpr int kTaylorTerms = 16;
// H: column-major with leading dimension ldh.  Leaves the result in S.
__device__ void block_expm(const double2* __restrict__ H, int ldh, int m, double dt, int imag, double2* A,
                           double2* P, double2* S, double2* T) {
    __shared__ int s_sq;
    const int t = threadIdx.x;
    const int mm = m * m;
    for (int o = t; o < mm; o += blockDim.x) {
        const int i = o % m, j = o / m;
        const double2 h = H[j * ldh + i];
        A[o] = imag ? make_double2(-dt * h.x, -dt * h.y)    // -dt h
                    : make_double2(dt * h.y, -dt * h.x);    // -i dt h
    }
    __syncthreads();
    // 1-norm: column sums by m threads (each in row order), then their maximum
    __shared__ double s_col[kMaxKrylov];
    if (t < m) {
        double c = 0.0;
        for (int i = 0; i < m; ++i) c += hypot(A[t * m + i].x, A[t * m + i].y);
        s_col[t] = c;
    }
    __syncthreads();
    if (t == 0) {
        double nrm = 0.0;
        for (int j = 0; j < m; ++j) nrm = fmax(nrm, s_col[j]);
        int sq = 0;
        while (nrm > 0.5 && sq < 60) {
            nrm *= 0.5;
            ++sq;
        }
        s_sq = sq;
    }
    __syncthreads();
    const double sc = ldexp(1.0, -s_sq);
    for (int o = t; o < mm; o += blockDim.x) {
        A[o].x *= sc;
        A[o].y *= sc;
        const int i = o % m, j = o / m;
        S[o] = make_double2(i == j ? 1.0 : 0.0, 0.0);
        P[o] = S[o];
    }
    __syncthreads();
    for (int k = 1; k <= kTaylorTerms; ++k) {
        // P <- P A / k
        const double ik = 1.0 / k;
        for (int o = t; o < mm; o += blockDim.x) {
            const int i = o % m, j = o / m;
            double x = 0.0, y = 0.0;
            for (int l = 0; l < m; ++l) {
                const double2 a = P[l * m + i], b = A[j * m + l];
                x += a.x * b.x - a.y * b.y;
                y += a.x * b.y + a.y * b.x;
            }
            T[o] = make_double2(x * ik, y * ik);
        }
        __syncthreads();
        for (int o = t; o < mm; o += blockDim.x) {
            P[o] = T[o];
            S[o].x += T[o].x;
            S[o].y += T[o].y;
        }
        __syncthreads();
    }
    for (int q = 0; q < s_sq; ++q) {
        for (int o = t; o < mm; o += blockDim.x) {
            const int i = o % m, j = o / m;
            double x = 0.0, y = 0.0;
            for (int l = 0; l < m; ++l) {
                const double2 a = S[l * m + i], b = S[j * m + l];
                x += a.x * b.x - a.y * b.y;
                y += a.x * b.y + a.y * b.x;
            }
            T[o] = make_double2(x, y);
        }
        __syncthreads();
        for (int o = t; o < mm; o += blockDim.x) S[o] = T[o];
        __syncthreads();
    }
}

struct TauLadder {
    double tau[kLadder];
};

// Block c evaluates E_c = exp(-i tau_c H_m) (imag: exp(-tau_c H_m)): writes
// its first column to col[c][0..m) and err[c].x = |h_{m+1,m}| |E_c[m-1][0]|
// (the error estimate divided by beta; 0 when exact is set, i.e. after a
// breakdown).
__global__ void expm_ladder_kernel(const double2* __restrict__ H, int ldh, int m, TauLadder taus, int exact,
                                   int imag, double2* __restrict__ col, double2* __restrict__ err) {
    __shared__ double2 A[kMaxKrylov * kMaxKrylov], P[kMaxKrylov * kMaxKrylov], S[kMaxKrylov * kMaxKrylov],
        T[kMaxKrylov * kMaxKrylov];
    const int c = blockIdx.x;
    block_expm(H, ldh, m, taus.tau[c], imag, A, P, S, T);
    for (int i = threadIdx.x; i < m; i += blockDim.x) col[c * kMaxKrylov + i] = S[i];
    if (threadIdx.x == 0) {
        const double2 hs = H[(m - 1) * ldh + m];
        const double2 e = S[m - 1];
        err[c] = make_double2(exact ? 0.0 : hypot(hs.x, hs.y) * hypot(e.x, e.y), 0.0);
    }
}

// ------------------------------------------------------------------- host
int launch_g_cell(const afem_mesh* m, const double* E, const double2* v, const double2* U, double2* z, int n,
                  cudaStream_t s, int velocity, const double2* U_hang = nullptr);

// The frozen mean fields at the hanging points, Uh[h] = sum_e w_e U[master_e]
// (the constraint rows C; the same products in the same order as the cell
// passes' own gather, so the cell pass gives the same bits either way), formed
// once per propagation instead of in every cell pass of every Krylov vector.
__global__ void hang_rows64_kernel(const double2* __restrict__ U, const int32_t* __restrict__ hp,
                                   const int32_t* __restrict__ hm, const double* __restrict__ hw, int64_t nh, int k,
                                   double2* __restrict__ Uh) {
    const int64_t n = nh * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x) {
        const int64_t h = o / k;
        const int c = int(o - h * k);
        double2 v = make_double2(0.0, 0.0);
        for (int e = hp[h]; e < hp[h + 1]; ++e) {
            const double2 u = U[int64_t(hm[e]) * k + c];
            v.x = fma(hw[e], u.x, v.x);
            v.y = fma(hw[e], u.y, v.y);
        }
        Uh[o] = v;
    }
}

__global__ void hang_rows32_kernel(const float2* __restrict__ U, const int32_t* __restrict__ hp,
                                   const int32_t* __restrict__ hm, const float* __restrict__ hw, int64_t nh, int k,
                                   float2* __restrict__ Uh) {
    const int64_t n = nh * k;
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x) {
        const int64_t h = o / k;
        const int c = int(o - h * k);
        float2 v = make_float2(0.0f, 0.0f);
        for (int e = hp[h]; e < hp[h + 1]; ++e) {
            const float2 u = U[int64_t(hm[e]) * k + c];
            v.x = fmaf(hw[e], u.x, v.x);
            v.y = fmaf(hw[e], u.y, v.y);
        }
        Uh[o] = v;
    }
}

template <typename TB>
int cdot_t(const double2* A, int na, const TB* B, int nb, const double* w, int64_t rows, int diag,
           double2* partial, double2* out, unsigned* counter, cudaStream_t s) {
    AFEM_LAUNCH((cdot_fused_kernel<TB>), red_blocks(), kRedThreads, 0, s, A, na, B, nb, w, rows, diag,
                reinterpret_cast<double*>(partial), counter, out);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int cdot(const double2* A, int na, const double2* B, int nb, const double* w, int64_t rows, int diag,
         double2* partial, double2* out, unsigned* counter, cudaStream_t s) {
    return cdot_t<double2>(A, na, B, nb, w, rows, diag, partial, out, counter, s);
}

__global__ void to_c64_kernel(const double2* __restrict__ x, float2* __restrict__ y, int64_t n) {
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x)
        y[o] = make_float2(narrow_f64(x[o].x), narrow_f64(x[o].y));
}

__global__ void narrow_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x)
        y[o] = narrow_f64(x[o]);
}

__global__ void widen_kernel(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n; o += int64_t(gridDim.x) * blockDim.x)
        y[o] = widen_f32(x[o]);
}

int convert_f64_f32(const double* x, float* y, int64_t n, cudaStream_t s) {
    if (n <= 0) return AFEM_OK;
    AFEM_LAUNCH((narrow_kernel), grid_for(n), 256, 0, s, x, y, n);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int convert_f32_f64(const float* x, double* y, int64_t n, cudaStream_t s) {
    if (n <= 0) return AFEM_OK;
    AFEM_LAUNCH((widen_kernel), grid_for(n), 256, 0, s, x, y, n);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int to_c64(const double2* x, float2* y, int64_t n, cudaStream_t s) {
    AFEM_LAUNCH((to_c64_kernel), grid_for(n), 256, 0, s, x, y, n);
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

int launch_g_cell32(const afem_mesh* m, const double* E, const float2* v, const float2* U, float2* z, int n,
                    cudaStream_t s, int velocity, const float2* U_hang = nullptr);

#define AFEM_NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

// One resident wave of kernel K (its occupancy per SM x the SMs), at most
// `cap` blocks: the FP64-bound Gram-Schmidt kernels then have no tail wave,
// and each thread covers more rows per FP64 block reduction.
template <auto K>
static unsigned wave_grid(unsigned cap) {
    static const int per_sm = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, kRedThreads, 0) != cudaSuccess || b < 1) b = 1;
        return b;
    }();
    const unsigned g = unsigned(device_sms() * per_sm);
    return g < cap ? g : cap;
}

// The Gram-Schmidt kernels for a run-time vector count nv (0 <= nv <= kMaxKrylov).
static int launch_krylov_dots(int nv, unsigned grid, cudaStream_t s, const double2* w, const double2* V,
                              int64_t stride, const double* ml, int64_t n_int, int n, const int* gate,
                              const double2* H, int ldh, const double2* beta2, double* partial, unsigned* counter,
                              double2* out) {
    switch (nv) {
        case 0:
            AFEM_LAUNCH((krylov_dots_kernel<0>), wave_grid<krylov_dots_kernel<0>>(grid), kRedThreads, 0, s, w, V,
                        stride, ml, n_int, n, gate, H, ldh,
                        beta2, partial, counter, out);
            break;
#define AFEM_DOTS_CASE(NVV)                                                                                       \
    case NVV:                                                                                                     \
        AFEM_LAUNCH((krylov_dots_kernel<NVV>), wave_grid<krylov_dots_kernel<NVV>>(grid), kRedThreads, 0, s, w, V, \
                    stride, ml, n_int, n, gate, H, ldh,                                                       \
                    beta2, partial, counter, out);                                                                \
        break;
            AFEM_NV_CASES(AFEM_DOTS_CASE)
#undef AFEM_DOTS_CASE
        default:
            return set_error(AFEM_EINVAL, "arnoldi: Krylov vector count out of range");
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

// The projector of G on the cell-pass output fused with the inner products
// against V_0..V_{nv-1}: complex64 z (precision form, phi32) or complex128 z.
static int launch_project_dots(int nv, unsigned grid, cudaStream_t s, const float2* z32, const float2* phi32,
                               const double2* z, const double2* phi, const double2* S, const DeviceMesh& D, int n,
                               double2* w, const double2* V, int64_t stride, const double2* H, int ldh,
                               const double2* beta2, double* partial, unsigned* counter, double2* out,
                               double* S_slots) {
    switch (nv) {
#define AFEM_PD_CASE(NVV)                                                                                           \
    case NVV:                                                                                                       \
        if (z32) {                                                                                                  \
            AFEM_LAUNCH((project32_dots_kernel<NVV>), wave_grid<project32_dots_kernel<NVV>>(grid), kRedThreads, 0, \
                        s, z32, phi32, S, D.ml_inv32, D.ml,                                                         \
                        D.n_interior, D.n_master, n, w, V, stride, H, ldh, beta2, partial, counter, out, S_slots);  \
        } else {                                                                                                    \
            AFEM_LAUNCH((project_dots_kernel<NVV>), wave_grid<project_dots_kernel<NVV>>(grid), kRedThreads, 0, s, \
                        z, phi, S, D.ml_inv, D.ml,                                                                  \
                        D.n_interior, D.n_master, n, w, V, stride, H, ldh, beta2, partial, counter, out);           \
        }                                                                                                           \
        break;
        AFEM_NV_CASES(AFEM_PD_CASE)
#undef AFEM_PD_CASE
        default:
            return set_error(AFEM_EINVAL, "arnoldi: Krylov vector count out of range");
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

static int launch_krylov_update(int nv, unsigned grid, cudaStream_t s, double2* w, const double2* V,
                                int64_t stride, const double2* c, const double* ml, int64_t n_int, int n,
                                const int* gate, int accumulate, double eta2, int* reorth, const double2* H, int ldh,
                                const double2* beta2, float2* w32, double* partial, unsigned* counter,
                                double2* Hcol) {
    switch (nv) {
#define AFEM_UPD_CASE(NVV)                                                                                      \
    case NVV:                                                                                                   \
        AFEM_LAUNCH((krylov_update_kernel<NVV>), wave_grid<krylov_update_kernel<NVV>>(grid), kRedThreads, 0, s, \
                    w, V, stride, c, ml, n_int, n, gate,                                                          \
                    accumulate, eta2, reorth, H, ldh, beta2, w32, partial, counter, Hcol);                      \
        break;
        AFEM_NV_CASES(AFEM_UPD_CASE)
#undef AFEM_UPD_CASE
        default:
            return set_error(AFEM_EINVAL, "arnoldi: Krylov vector count out of range");
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

// substep_close_kernel for m = 0 (open the first substep from src) or the
// substep's Krylov dimension m (1..kMaxKrylov).
static int launch_substep_close(int m, unsigned grid, cudaStream_t s, double2* V, int64_t stride, const double2* y,
                                double scale, const double2* H, int ldh, double2* beta2, const double2* src,
                                const DeviceMesh& D, int n, double2* out, float2* v32, double* partial,
                                unsigned* counter) {
    switch (m) {
        case 0:
            AFEM_LAUNCH((substep_close_kernel<0>), wave_grid<substep_close_kernel<0>>(grid), kRedThreads, 0, s, V,
                        stride, y, scale, H, ldh, beta2, src, D.ml, D.n_interior, D.n_master, n, out, v32, partial,
                        counter, beta2);
            break;
#define AFEM_CLOSE_CASE(MM)                                                                                   \
    case MM:                                                                                                  \
        AFEM_LAUNCH((substep_close_kernel<MM>), wave_grid<substep_close_kernel<MM>>(grid), kRedThreads, 0, s, \
                    V, stride, y, scale, H, ldh, beta2, src, D.ml, D.n_interior, D.n_master, n, out, v32,      \
                    partial, counter, beta2);                                                                 \
        break;
            AFEM_NV_CASES(AFEM_CLOSE_CASE)
#undef AFEM_CLOSE_CASE
        default:
            return set_error(AFEM_EINVAL, "arnoldi: Krylov dimension out of range");
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

static unsigned rowcol_grid(int64_t rows, int n) {
    const int64_t R = kRedThreads / n;
    int64_t g = (rows + R - 1) / R;
    if (g < 1) g = 1;
    if (g > red_blocks()) g = red_blocks();
    return unsigned(g);
}

// The cell pass of G and the projector overlaps S[j][p] = phi_j^H z_p (equal to
// phi_j^H M_L y_p); the projector itself runs fused with the first
// Gram-Schmidt pass.  Precision form: the cell pass in complex64 from v32 (the
// complex64 copy of the vector) and the overlaps from phi32.
static int g_cell_overlaps32(afem_mesh* m, const double* E, const float2* phi32, const float2* U32, int n,
                             const float2* v32, ArnoldiWork& w, cudaStream_t s, int velocity) {
    const DeviceMesh& D = m->dev;
    int rc;
    {   // algorithmic bytes: read v, U (n^2 fields), write z, complex64
        ProfScope ps(AFEM_PROF_GCELL32, s, double(D.n_master) * 8.0 * n * (2 + n));
        rc = w.gb ? launch_g_cell32_blocks(m, v32, w.gb, w.z32, n, w.bulk_err, w.vh32, s)
                  : launch_g_cell32(m, E, v32, U32, w.z32, n, s, velocity, w.uh32);
        if (rc) return rc;
    }
    auto* part = reinterpret_cast<double*>(w.cpartial);
    switch (n) {
#define AFEM_OV_CASE(NO)                                                                                        \
    case NO:                                                                                                    \
        AFEM_LAUNCH((overlap32_kernel<NO>), red_blocks(), kRedThreads, 0, s, phi32, w.z32, D.n_interior,         \
                    w.Sslots);                                                                                  \
        break;
        AFEM_OV_CASE(1)
        AFEM_OV_CASE(2)
        AFEM_OV_CASE(3)
        AFEM_OV_CASE(4)
        AFEM_OV_CASE(5)
        AFEM_OV_CASE(6)
        AFEM_OV_CASE(7)
        AFEM_OV_CASE(8)
#undef AFEM_OV_CASE
        default:
            return set_error(AFEM_EINVAL, "arnoldi: orbital count out of range");
    }
    AFEM_CUDA_TRY(cudaGetLastError());
    return AFEM_OK;
}

static int g_cell_overlaps(afem_mesh* m, const double* E, const double2* phi, const double2* U, int n,
                           const double2* v, ArnoldiWork& w, cudaStream_t s, int velocity) {
    const DeviceMesh& D = m->dev;
    int rc;
    {
        const int p1 = D.p + 1;
        ProfScope ps(AFEM_PROF_CELL64, s, double(D.ncell) * p1 * p1 * p1 * 2.0 * n * (3.0 * p1 * 2.0 + 6.0));
        rc = launch_g_cell(m, E, v, U, w.z, n, s, velocity, w.uh);
    }
    if (rc) return rc;
    return cdot(phi, n, w.z, n, nullptr, D.n_interior, 0, w.cpartial, w.S, w.counters, s);
}

int arnoldi_reserve(afem_mesh* m, int n, int mk, ArnoldiWork& w) {
    const size_t NV = size_t(m->dev.n_master) * n;
    auto carve = [&](Carver& cv) {
        w.V = cv.take<double2>(size_t(mk + 1) * NV);
        w.z = cv.take<double2>(NV);
        w.cpartial = cv.take<double2>(size_t(kRedBlocksMax) * 256);
        w.S = cv.take<double2>(kMaxOrbProj * kMaxOrbProj);
        w.Sslots = cv.take<double>(size_t(kOvSlots) * 2 * kMaxOrbProj * kMaxOrbProj);
        w.res = cv.take<double2>(kResSize);
        w.c1 = cv.take<double2>(kMaxKrylov + 1);
        w.c2 = cv.take<double2>(kMaxKrylov + 1);
        w.v32 = cv.take<float2>(NV);
        w.z32 = cv.take<float2>(NV);
        w.phi32 = cv.take<float2>(NV);
        w.U32 = cv.take<float2>(NV * n);
        w.Uh = cv.take<double2>(size_t(m->dev.n_hanging) * n * n);
        w.Uh32 = cv.take<float2>(size_t(m->dev.n_hanging) * n * n);
        w.vh32 = reinterpret_cast<float4*>(cv.take<float2>(size_t(m->dev.n_hanging) * n + 2));
        w.counters = cv.take<unsigned>(4);
        w.flag = cv.take<int>(4);
    };
    Carver measure(nullptr);
    carve(measure);
    int rc = m->ws_arnoldi.reserve(measure.size());
    if (rc) return rc;
    Carver cv(m->ws_arnoldi.ptr);
    carve(cv);
    w.stride = int64_t(NV);
    w.H = w.res + kResH;
    w.beta2 = w.res + kResBeta2;
    w.col = w.res + kResCol;
    w.err = w.res + kResErr;
    w.bulk_err = reinterpret_cast<double*>(w.res + kResFlag);
    w.gb = nullptr;
    return AFEM_OK;
}

// Candidate substep lengths of one ladder: tau_max * 2^(-c/8), c = 0..K-1.
static TauLadder make_ladder(double tau_max, int K) {
    TauLadder L{};
    for (int c = 0; c < kLadder; ++c) L.tau[c] = c < K ? tau_max * std::pow(2.0, -kLadderLog2 * c) : 0.0;
    return L;
}

// Propagates phi by exp(-i G dt) with G frozen at phi (projector), U and E.
// tol <= 0: one Krylov step of dimension mk over the whole dt.  tol > 0:
// substeps from fresh Krylov spaces of the same G, each as long as the error
// estimate beta |h_{m+1,m}| |e_m^T exp(-i tau H_m) e_1| <= tol * beta allows
// among the candidates tau_max 2^(-c/8), c = 0..63, where tau_max is the
// remainder for the first substep and min(remainder, 2 tau_previous) after
// it; when no candidate passes, the ladder continues below the smallest one
// (the paper fixes the Krylov accuracy by such an estimate; here the
// dimension is fixed and the substep adapts).
int arnoldi_step(afem_mesh* m, const double* E, const double2* phi, const double2* U, const float2* U32, int n,
                 int mk, double dt, int mixed, double tol, double2* phi_out, double* err_est, int* m_used_out,
                 int* breakdown_out, int* substeps_out, cudaStream_t s, int flags, int adaptive_steps,
                 int* dim_sum_out, int* unmet_out) {
    const DeviceMesh& D = m->dev;
    if (mk < 1 || mk > kMaxKrylov) return set_error(AFEM_EINVAL, "arnoldi: krylov_m out of range");
    if (n < 1 || n > kMaxOrbProj) return set_error(AFEM_EINVAL, "arnoldi: orbital count out of range");
    if (adaptive_steps < 0 || (adaptive_steps > 0 && !(tol > 0.0)))
        return set_error(AFEM_EINVAL, "arnoldi: the adaptive dimension needs steps >= 1 and a threshold > 0");
    const int imag = (flags & kArnImaginary) ? 1 : 0;
    const int velocity = (flags & kArnVelocity) ? 1 : 0;   // E holds the vector potential A
    const bool adaptive = adaptive_steps > 0;
    const double tau_fixed = adaptive ? dt / adaptive_steps : 0.0;
    ArnoldiWork w{};
    int rc = arnoldi_reserve(m, n, mk, w);
    if (rc) return rc;
    const int64_t NV = w.stride;
    const bool projector = !(flags & kArnNoProjector);
    // candidate exponentials exp(-i tau H_m), or exp(+i tau H_m) propagating backward
    auto signed_ladder = [&](double tm, int K) {
        TauLadder L = make_ladder(tm, K);
        if (flags & kArnBackward)
            for (int c = 0; c < kLadder; ++c) L.tau[c] = -L.tau[c];
        return L;
    };
    if (!projector) AFEM_CUDA_TRY(cudaMemsetAsync(w.S, 0, sizeof(double2) * kMaxOrbProj * kMaxOrbProj, s));
    if (mixed) {
        if (U && !U32) {
            if ((rc = to_c64(U, w.U32, D.n_master * n * n, s))) return rc;
            U32 = w.U32;
        }
        if ((rc = to_c64(phi, w.phi32, NV, s))) return rc;
    }
    w.uh = nullptr;
    w.uh32 = nullptr;
    if (D.n_hanging > 0 && (mixed ? U32 != nullptr : U != nullptr)) {
        const int64_t nh = D.n_hanging;
        const int k = n * n;
        if (mixed) {
            AFEM_LAUNCH((hang_rows32_kernel), grid_for(nh * k), 256, 0, s, U32, D.hang_ptr, D.hang_master,
                        D.hang_w32, nh, k, w.Uh32);
            w.uh32 = w.Uh32;
        } else {
            AFEM_LAUNCH((hang_rows64_kernel), grid_for(nh * k), 256, 0, s, U, D.hang_ptr, D.hang_master, D.hang_w,
                        nh, k, w.Uh);
            w.uh = w.Uh;
        }
        AFEM_CUDA_TRY(cudaGetLastError());
    }
    w.gb = nullptr;
    if (mixed && U32 && gcell_blocks_apply(m, n, velocity)) {
        // the frozen pointwise part of G, one contiguous block per cell, staged by
        // the cell pass with one bulk copy (formed once for all substeps)
        if ((rc = m->ws_gblocks.reserve(gcell_blocks_bytes(m, n)))) return rc;
        auto* B = static_cast<float4*>(m->ws_gblocks.ptr);
        if ((rc = build_gcell_blocks32(m, E, U32, w.uh32, n, B, s))) return rc;
        w.gb = B;
        AFEM_CUDA_TRY(cudaMemsetAsync(w.bulk_err, 0, sizeof(double), s));
    }
    AFEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned), s));
    AFEM_CUDA_TRY(cudaMemsetAsync(w.flag, 0, 4 * sizeof(int), s));
    AFEM_CUDA_TRY(cudaMemsetAsync(w.Sslots, 0, sizeof(double) * kOvSlots * 2 * kMaxOrbProj * kMaxOrbProj, s));
    const int ldh = kMaxKrylov + 1;
    const unsigned gdots = rowcol_grid(D.n_interior, n);
    const unsigned gproj = rowcol_grid(D.n_master, n);
    double* part = reinterpret_cast<double*>(w.cpartial);
    unsigned* cnt = w.counters + 1;
    const double eta2 = 1e-4;   // second pass when the update left less than 1e-2 of the norm
    double remaining = dt, tau_prev = 0.0;
    double err_sum = 0.0;
    int substeps = 0, m_used = mk, brk = 0, dim_max = 0, dim_sum = 0, unmet = 0;
    std::vector<double2> res(kResSize);
    auto fetch = [&]() -> int {
        AFEM_CUDA_TRY(cudaMemcpyAsync(res.data(), w.res, kResSize * sizeof(double2), cudaMemcpyDeviceToHost, s));
        AFEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (w.gb && res[kResFlag].x != 0.0)
            return set_error(AFEM_ECUDA, "arnoldi: a G cell pass gave up waiting for a per-cell block copy");
        return AFEM_OK;
    };
    float2* v32 = mixed ? w.v32 : nullptr;
    // V_0 = phi (unscaled), its complex64 copy and beta^2 = <phi, phi>_M; later
    // substeps get theirs from the closing pass of the previous one
    if ((rc = launch_substep_close(0, gproj, s, w.V, NV, nullptr, 0.0, w.H, ldh, w.beta2, phi, D, n, nullptr, v32,
                                   part, cnt)))
        return rc;
    while (remaining > 0.0) {
        if (substeps >= 4096) return set_error(AFEM_EINVAL, "arnoldi: more than 4096 substeps (tolerance too tight)");
        AFEM_CUDA_TRY(cudaMemsetAsync(w.H, 0, sizeof(double2) * ldh * kMaxKrylov, s));
        for (int j = 0; j < mk; ++j) {
            double2* Wn = w.V + (j + 1) * NV;
            double2* Hcol = w.H + j * ldh;
            // w = G q_j (the cell pass on the stored V_j, scaled in the projector
            // pass) with the inner products against q_0..q_j, the update (which
            // leaves V_{j+1} = h_{j+1,j} q_{j+1}), and a second pass when the
            // update cancelled most of w
            if (!projector) {   // the cell pass alone; S stays zero
                if (mixed) {
                    rc = w.gb ? launch_g_cell32_blocks(m, w.v32, w.gb, w.z32, n, w.bulk_err, w.vh32, s)
                              : launch_g_cell32(m, E, w.v32, U32, w.z32, n, s, velocity, w.uh32);
                    if (rc) return rc;
                } else {
                    if ((rc = launch_g_cell(m, E, w.V + j * NV, U, w.z, n, s, velocity, w.uh))) return rc;
                }
            } else if (mixed) {
                if ((rc = g_cell_overlaps32(m, E, w.phi32, U32, n, w.v32, w, s, velocity))) return rc;
            } else {
                if ((rc = g_cell_overlaps(m, E, phi, U, n, w.V + j * NV, w, s, velocity))) return rc;
            }
            // algorithmic FP64 flops per element: 8 per basis vector in each pass
            // (one complex multiply-add), plus 4 for the new norm in the update
            const double gs_flops = double(D.n_interior) * n * 8.0 * (j + 1);
            {
                ProfScope ps(AFEM_PROF_GS, s, gs_flops);
                rc = launch_project_dots(j + 1, gproj, s, mixed ? w.z32 : nullptr, w.phi32, w.z, phi, w.S, D, n, Wn,
                                         w.V, NV, w.H, ldh, w.beta2, part, cnt, w.c1,
                                         (mixed && projector) ? w.Sslots : nullptr);
            }
            if (!rc) {
                ProfScope ps(AFEM_PROF_GS, s, gs_flops + double(D.n_interior) * n * 4.0);
                rc = launch_krylov_update(j + 1, gdots, s, Wn, w.V, NV, w.c1, D.ml, D.n_interior, n, nullptr, 0, eta2,
                                          w.flag, w.H, ldh, w.beta2, v32, part, cnt, Hcol);
            }
            if (rc ||
                (rc = launch_krylov_dots(j + 1, gdots, s, Wn, w.V, NV, D.ml, D.n_interior, n, w.flag, w.H, ldh,
                                         w.beta2, part, cnt, w.c2)) ||
                (rc = launch_krylov_update(j + 1, gdots, s, Wn, w.V, NV, w.c2, D.ml, D.n_interior, n, w.flag, 1,
                                           eta2, nullptr, w.H, ldh, w.beta2, v32, part, cnt, Hcol)))
                return rc;
            if (adaptive) {
                // Sec. 3.2's rule: the estimate of dimension j + 1 at the fixed step;
                // the first dimension that meets the threshold (or breaks down) ends
                // the process
                AFEM_LAUNCH((expm_ladder_kernel), 1, 256, 0, s, w.H, ldh, j + 1, signed_ladder(tau_fixed, 1), 0,
                            imag, w.col, w.err);
                AFEM_CUDA_TRY(cudaGetLastError());
                if ((rc = fetch())) return rc;
                const double b = std::sqrt(res[kResBeta2].x);
                const double hn = res[kResH + j * ldh + j + 1].x;
                if (!(b > 0.0) || !std::isfinite(b) || !std::isfinite(hn))
                    return set_error(AFEM_ENAN, "arnoldi: zero or non-finite Krylov vector");
                m_used = j + 1;
                brk = hn < 1e-14 * b ? 1 : 0;
                if (brk || res[kResErr].x <= tol) break;
            }
        }
        double tau, err;
        int pick = 0;
        if (adaptive) {
            const double beta = std::sqrt(res[kResBeta2].x);
            tau = tau_fixed;
            err = brk ? 0.0 : beta * res[kResErr].x;
            if (!brk && res[kResErr].x > tol) ++unmet;
            if ((rc = launch_substep_close(m_used, gproj, s, w.V, NV, w.col, beta, w.H, ldh, w.beta2, nullptr, D, n,
                                           phi_out, v32, part, cnt)))
                return rc;
            err_sum += err;
            ++substeps;
            dim_max = std::max(dim_max, m_used);
            dim_sum += m_used;
            tau_prev = tau;
            remaining = substeps >= adaptive_steps ? 0.0 : remaining - tau;
            continue;
        }
        // candidate substeps, one block each; a single host wait per ladder
        double tau_max = (tol <= 0.0 || substeps == 0) ? remaining : std::fmin(remaining, 2.0 * tau_prev);
        int K = tol <= 0.0 ? 1 : kLadder;
        int exact = 0;
        AFEM_LAUNCH((expm_ladder_kernel), K, 256, 0, s, w.H, ldh, mk, signed_ladder(tau_max, K), 0, imag, w.col,
                    w.err);
        AFEM_CUDA_TRY(cudaGetLastError());
        if ((rc = fetch())) return rc;
        const double beta = std::sqrt(res[kResBeta2].x);
        if (!(beta > 0.0) || !std::isfinite(beta)) return set_error(AFEM_ENAN, "arnoldi: zero or non-finite norm");
        m_used = mk;
        brk = 0;
        for (int j = 0; j < mk; ++j) {
            const double hn = res[kResH + j * ldh + j + 1].x;
            if (!std::isfinite(hn)) return set_error(AFEM_ENAN, "arnoldi: non-finite Krylov vector");
            if (hn < 1e-14 * beta) {
                m_used = j + 1;
                brk = 1;
                break;
            }
        }
        if (brk) {   // invariant subspace: the projected exponential is exact
            tau_max = remaining;
            K = 1;
            exact = 1;
            AFEM_LAUNCH((expm_ladder_kernel), 1, 256, 0, s, w.H, ldh, m_used, signed_ladder(tau_max, 1), 1, imag,
                        w.col, w.err);
            AFEM_CUDA_TRY(cudaGetLastError());
            if ((rc = fetch())) return rc;
        }
        pick = -1;
        for (int round = 0;; ++round) {
            for (int c = 0; c < K; ++c) {
                if (exact || tol <= 0.0 || res[kResErr + c].x <= tol) {
                    pick = c;
                    break;
                }
            }
            if (pick >= 0) break;
            if (round >= 8) {   // accept the smallest candidate
                pick = K - 1;
                break;
            }
            tau_max *= std::pow(2.0, -kLadderLog2 * K);
            AFEM_LAUNCH((expm_ladder_kernel), K, 256, 0, s, w.H, ldh, m_used, signed_ladder(tau_max, K), 0, imag,
                        w.col, w.err);
            AFEM_CUDA_TRY(cudaGetLastError());
            if ((rc = fetch())) return rc;
        }
        tau = make_ladder(tau_max, K).tau[pick];
        err = beta * res[kResErr + pick].x;
        // phi_out = beta V_m exp(-i tau H_m) e_1, which also opens the next substep
        if ((rc = launch_substep_close(m_used, gproj, s, w.V, NV, w.col + pick * kMaxKrylov, beta, w.H, ldh, w.beta2,
                                       nullptr, D, n, phi_out, v32, part, cnt)))
            return rc;
        err_sum += err;
        ++substeps;
        dim_max = std::max(dim_max, m_used);
        dim_sum += m_used;
        tau_prev = tau;
        remaining = (tau >= remaining) ? 0.0 : remaining - tau;
    }
    AFEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (err_est) *err_est = err_sum;
    if (m_used_out) *m_used_out = adaptive ? dim_max : m_used;
    if (dim_sum_out) *dim_sum_out = dim_sum;
    if (unmet_out) *unmet_out = unmet;
    if (breakdown_out) *breakdown_out = brk;
    if (substeps_out) *substeps_out = substeps;
    return AFEM_OK;
}

}  // namespace afem
