// Arnoldi workspace layout and the G-operator entry points shared by the
// Arnoldi step and the MCTDHF step.
#pragma once

#include "afem_internal.h"

namespace afem {

constexpr int kMaxKrylov = 16;
constexpr int kLadder = 64;             // candidate substep lengths evaluated per ladder
constexpr double kLadderLog2 = 0.125;   // candidate c is tau_max * 2^(-c kLadderLog2)
constexpr int kMaxOrbProj = 8;   // orbitals (the C ABI accepts 1..8)

// Small results the host reads once per substep, contiguous in device memory:
// the Hessenberg matrix, beta^2, the first columns of the candidate
// exponentials and their error estimates (over beta, in .x).
constexpr int kResH = 0;
constexpr int kResBeta2 = (kMaxKrylov + 1) * kMaxKrylov;
constexpr int kResCol = kResBeta2 + 1;
constexpr int kResErr = kResCol + kLadder * kMaxKrylov;
constexpr int kResFlag = kResErr + kLadder;   // .x != 0: a G cell pass gave up waiting for a block copy
constexpr int kResSize = kResFlag + 1;

struct ArnoldiWork {
    double2* V;          // [m+1][N][n] Krylov basis
    double2* z;          // [N][n] cell-pass output
    double2* cpartial;   // reduction partials
    double2* S;          // [n][n] projector overlaps
    double* Sslots;      // [16][2 n^2] FP64 slots of the precision form's overlaps (summed by the projector)
    double2* res;        // kResSize small results (below)
    double2* H;          // (kMaxKrylov+1) x kMaxKrylov Hessenberg, column-major (in res)
    double2* beta2;      // <phi, phi>_M of the substep's start vector (in res)
    double2* col;        // [kLadder][kMaxKrylov] first columns of exp(-i tau_c H_m) (in res)
    double2* err;        // [kLadder] error estimates over beta (in res)
    double2* c1;         // inner products and norm of the first Gram-Schmidt pass
    double2* c2;         // the same for the second pass
    float2* v32;         // [N][n] complex64 copy of the vector G is applied to (mixed form)
    float2* z32;         // [N][n] complex64 cell-pass output (mixed form)
    float2* phi32;       // [N][n] complex64 copy of the frozen orbitals (mixed-form projector)
    float2* U32;         // [N][n][n] complex64 mean-field fields (mixed form)
    double2* Uh;         // [nh][n][n] the mean fields at the hanging points (C U), FP64 cell pass
    float2* Uh32;        // [nh][n][n] the same in complex64
    const double2* uh;   // Uh once formed for this call, else null (interpolated in every cell pass)
    const float2* uh32;
    unsigned* counters;  // last-block reduction counters (zeroed per call)
    int* flag;           // second-pass flag
    const float4* gb;    // frozen per-cell blocks of the G cell pass for this call, else null
    float4* vh32;        // [nh][n/2] C v at the hanging points (pipelined G cell pass)
    double* bulk_err;    // res[kResFlag].x
    int64_t stride;      // N * n
};

int cdot(const double2* A, int na, const double2* B, int nb, const double* w, int64_t rows, int diag,
         double2* partial, double2* out, unsigned* counter, cudaStream_t s);
// flags: kArnNoProjector applies H1~ + mean field without the projector Q
// (the one-electron Schroedinger propagator and its block Frechet form);
// kArnBackward propagates by exp(+i G dt); kArnImaginary by exp(-G dt)
// (imaginary time).  adaptive_steps > 0: the rule of Sec. 3.2 -- dt split
// into adaptive_steps equal steps, each with the smallest Krylov dimension
// (<= mk) whose estimate is <= tol beta (mk when none is); dim_sum_out then
// receives the summed dimensions, m_used_out the largest and unmet_out the
// number of steps whose estimate stayed above the threshold at mk.
constexpr int kArnNoProjector = 1;
constexpr int kArnBackward = 2;
constexpr int kArnImaginary = 4;
constexpr int kArnVelocity = 8;   // velocity gauge: the field argument is the vector potential A
int arnoldi_step(afem_mesh* m, const double* E, const double2* phi, const double2* U, const float2* U32, int n,
                 int mk, double dt, int mixed, double tol, double2* phi_out, double* err_est, int* m_used_out,
                 int* breakdown_out, int* substeps_out, cudaStream_t s, int flags = 0, int adaptive_steps = 0,
                 int* dim_sum_out = nullptr, int* unmet_out = nullptr);
int to_c64(const double2* x, float2* y, int64_t n, cudaStream_t s);

}  // namespace afem
