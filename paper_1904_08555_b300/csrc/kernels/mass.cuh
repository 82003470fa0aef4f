// mass.cuh -- mass operator of tensor-product finite elements, the Laghos
// kernel of Sec. 5 whose specializations are keyed on the dimension, the
// dofs per dimension D and the quadrature points per dimension Q:
//
//     y_e = B^T diag(op_e) B x_e,   B = B1 (x) B1 [(x) B1],   every element e,
//
// with B1[q][d] the 1-D basis at the quadrature points (Q x D, row-major), x_e
// and y_e D^DIM values, op_e Q^DIM values, first index fastest.  Evaluated by
// sum factorization: one 1-D contraction per dimension on the way to the
// quadrature points, the pointwise scaling, one per dimension back.
//
// Thread layout: an element owns a square of M x M threads (M = max(D, Q));
// thread (tx, ty) computes the entries of each stage indexed by (tx, ty),
// looping over the third index in 3-D.  A block holds EPB elements, each with
// two shared-memory buffers of M^DIM values that the stages alternate
// between, and B1 once.  Every thread of a block takes every barrier.
#ifndef CJ_MASS_CUH
#define CJ_MASS_CUH
#include "geometry.h"

namespace cj {

__device__ __forceinline__ double mass_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mass_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// One element's stages.  D, Q, DIM are compile-time in the specialized kernel
// and run-time in the generic one (the loops below are the same code; with
// constants the compiler unrolls them).  b: B1 in shared memory (Q x D);
// u, v: the element's two buffers (M^DIM each); tx, ty < M.
template <class T, class Int>
__device__ __forceinline__ void mass_element(const T* __restrict__ x, const T* __restrict__ op, T* __restrict__ y,
                                             const T* b, T* u, T* v, Int DIM, Int D, Int Q, Int M, int tx, int ty,
                                             bool active) {
    // buffers are indexed [k][j][i] with i fastest, extents M
    if (DIM == 2) {
        // X[jy][jx] -> u
        if (active && tx < D && ty < D) u[ty * M + tx] = x[ty * D + tx];
        __syncthreads();
        // T1[jy][qx] = sum_jx B1[qx][jx] X[jy][jx] -> v   (thread qx = tx, jy = ty)
        if (active && tx < Q && ty < D) {
            T s = T(0);
#pragma unroll
            for (Int jx = 0; jx < D; ++jx) s = mass_fma(b[tx * D + jx], u[ty * M + jx], s);
            v[ty * M + tx] = s;
        }
        __syncthreads();
        // T2[qy][qx] = op * sum_jy B1[qy][jy] T1[jy][qx] -> u   (qx = tx, qy = ty)
        if (active && tx < Q && ty < Q) {
            T s = T(0);
#pragma unroll
            for (Int jy = 0; jy < D; ++jy) s = mass_fma(b[ty * D + jy], v[jy * M + tx], s);
            u[ty * M + tx] = op[ty * Q + tx] * s;
        }
        __syncthreads();
        // T3[qy][jx] = sum_qx B1[qx][jx] T2[qy][qx] -> v   (jx = tx, qy = ty)
        if (active && tx < D && ty < Q) {
            T s = T(0);
#pragma unroll
            for (Int qx = 0; qx < Q; ++qx) s = mass_fma(b[qx * D + tx], u[ty * M + qx], s);
            v[ty * M + tx] = s;
        }
        __syncthreads();
        // Y[jy][jx] = sum_qy B1[qy][jy] T3[qy][jx]   (jx = tx, jy = ty)
        if (active && tx < D && ty < D) {
            T s = T(0);
#pragma unroll
            for (Int qy = 0; qy < Q; ++qy) s = mass_fma(b[qy * D + ty], v[qy * M + tx], s);
            y[ty * D + tx] = s;
        }
    } else {
        const Int MM = M * M;
        // X[jz][jy][jx] -> u
        if (active && tx < D && ty < D)
#pragma unroll
            for (Int jz = 0; jz < D; ++jz) u[jz * MM + ty * M + tx] = x[(jz * D + ty) * D + tx];
        __syncthreads();
        // x: T1[jz][jy][qx] = sum_jx B1[qx][jx] X[jz][jy][jx] -> v   (qx = tx, jy = ty)
        if (active && tx < Q && ty < D)
#pragma unroll
            for (Int jz = 0; jz < D; ++jz) {
                T s = T(0);
#pragma unroll
                for (Int jx = 0; jx < D; ++jx) s = mass_fma(b[tx * D + jx], u[jz * MM + ty * M + jx], s);
                v[jz * MM + ty * M + tx] = s;
            }
        __syncthreads();
        // y: T2[jz][qy][qx] = sum_jy B1[qy][jy] T1[jz][jy][qx] -> u   (qx = tx, qy = ty)
        if (active && tx < Q && ty < Q)
#pragma unroll
            for (Int jz = 0; jz < D; ++jz) {
                T s = T(0);
#pragma unroll
                for (Int jy = 0; jy < D; ++jy) s = mass_fma(b[ty * D + jy], v[jz * MM + jy * M + tx], s);
                u[jz * MM + ty * M + tx] = s;
            }
        __syncthreads();
        // z, scaling, z back, on thread (qx, qy)'s own line:
        // T3[qz] = op[qz][qy][qx] sum_jz B1[qz][jz] T2[jz]; T4[jz] = sum_qz B1[qz][jz] T3[qz] -> v
        if (active && tx < Q && ty < Q) {
            for (Int jz = 0; jz < D; ++jz) v[jz * MM + ty * M + tx] = T(0);
#pragma unroll
            for (Int qz = 0; qz < Q; ++qz) {
                T s = T(0);
#pragma unroll
                for (Int jz = 0; jz < D; ++jz) s = mass_fma(b[qz * D + jz], u[jz * MM + ty * M + tx], s);
                s = op[(qz * Q + ty) * Q + tx] * s;
#pragma unroll
                for (Int jz = 0; jz < D; ++jz)
                    v[jz * MM + ty * M + tx] = mass_fma(b[qz * D + jz], s, v[jz * MM + ty * M + tx]);
            }
        }
        __syncthreads();
        // y back: T5[jz][jy][qx] = sum_qy B1[qy][jy] T4[jz][qy][qx] -> u   (qx = tx, jy = ty)
        if (active && tx < Q && ty < D)
#pragma unroll
            for (Int jz = 0; jz < D; ++jz) {
                T s = T(0);
#pragma unroll
                for (Int qy = 0; qy < Q; ++qy) s = mass_fma(b[qy * D + ty], v[jz * MM + qy * M + tx], s);
                u[jz * MM + ty * M + tx] = s;
            }
        __syncthreads();
        // x back: Y[jz][jy][jx] = sum_qx B1[qx][jx] T5[jz][jy][qx]   (jx = tx, jy = ty)
        if (active && tx < D && ty < D)
#pragma unroll
            for (Int jz = 0; jz < D; ++jz) {
                T s = T(0);
#pragma unroll
                for (Int qx = 0; qx < Q; ++qx) s = mass_fma(b[qx * D + tx], u[jz * MM + ty * M + qx], s);
                y[(jz * D + ty) * D + tx] = s;
            }
    }
}

// Specialized: DIM, D, Q and the elements per block are template arguments.
// Block: EPB * M * M threads; thread t works on element t / (M M) of the
// block, at (tx, ty) = ((t % M M) % M, (t % M M) / M).
template <class T, int DIM, int D, int Q, int EPB>
__global__ void __launch_bounds__(cjg::mass_threads(D, Q, EPB))
mass_apply(const T* __restrict__ B1, const T* __restrict__ op, const T* __restrict__ x, T* __restrict__ y,
           long long ne) {
    constexpr int M = D > Q ? D : Q;
    constexpr int ND = DIM == 2 ? D * D : D * D * D, NQ = DIM == 2 ? Q * Q : Q * Q * Q;
    constexpr int MD = DIM == 2 ? M * M : M * M * M;
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* b = reinterpret_cast<T*>(cj_smem);
    T* bufs = b + cjg::mass_b_elems(D, Q);
    const int t = threadIdx.x, le = t / (M * M), r = t - le * M * M;
    for (int i = t; i < Q * D; i += cjg::mass_threads(D, Q, EPB)) b[i] = B1[i];
    const long long e = (long long)blockIdx.x * EPB + le;
    // threads past EPB elements (the block is rounded up to whole warps) only take the barriers
    const bool active = le < EPB && e < ne;
    const long long ec = active ? e : 0;
    const int lb = le < EPB ? le : 0;
    mass_element<T, int>(x + ec * ND, op + ec * NQ, y + ec * ND, b, bufs + (2 * lb) * MD, bufs + (2 * lb + 1) * MD,
                         DIM, D, Q, M, r % M, r / M, active);
}

// One element (T = 4 or 8 bytes) from global to shared memory without
// registers: completes at the next cp.async.wait_group that covers it.
template <class T>
__device__ __forceinline__ void mass_cp_async(T* dst, const T* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

// Specialized and persistent (tile {EPB, 1, 0, 0}): block b takes element
// groups b, b + grid, ... (EPB consecutive elements each).  While one group
// is computed, the x and op values of the block's next group are copied into
// the other of two shared-memory stages with cp.async, so that each SM keeps
// loads in flight through the compute stages.  Shared memory: B1, the two
// work buffers per element, then stage s at [x: EPB D^dim | op: EPB Q^dim].
template <class T, int DIM, int D, int Q, int EPB>
__global__ void __launch_bounds__(cjg::mass_threads(D, Q, EPB))
mass_apply_pipe(const T* __restrict__ B1, const T* __restrict__ op, const T* __restrict__ x, T* __restrict__ y,
                long long ne) {
    constexpr int M = D > Q ? D : Q;
    constexpr int ND = DIM == 2 ? D * D : D * D * D, NQ = DIM == 2 ? Q * Q : Q * Q * Q;
    constexpr int MD = DIM == 2 ? M * M : M * M * M;
    constexpr int NT = cjg::mass_threads(D, Q, EPB);
    constexpr int SX = EPB * ND, SO = EPB * NQ;   // stage extents
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* b = reinterpret_cast<T*>(cj_smem);
    T* bufs = b + cjg::mass_b_elems(D, Q);
    T* stage = bufs + 2 * EPB * MD;
    const int t = threadIdx.x, le = t / (M * M), r = t - le * M * M;
    for (int i = t; i < Q * D; i += NT) b[i] = B1[i];
    const long long ngroups = (ne + EPB - 1) / EPB;
    // the x and op values of group g (cnt elements, contiguous in both) into stage s
    auto issue = [&](long long g, int s) {
        const long long e0 = g * EPB;
        const int cnt = ne - e0 < EPB ? (int)(ne - e0) : EPB;
        T* sx = stage + s * (SX + SO);
        T* so = sx + SX;
        for (int i = t; i < cnt * ND; i += NT) mass_cp_async(sx + i, x + e0 * ND + i);
        for (int i = t; i < cnt * NQ; i += NT) mass_cp_async(so + i, op + e0 * NQ + i);
    };
    if ((long long)blockIdx.x < ngroups) issue(blockIdx.x, 0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    int s = 0;
    for (long long g = blockIdx.x; g < ngroups; g += gridDim.x, s ^= 1) {
        // the next group's copies start before this group's wait
        if (g + gridDim.x < ngroups) issue(g + gridDim.x, s ^ 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // this group's stage has landed
        __syncthreads();
        const long long e = g * EPB + le;
        const bool active = le < EPB && e < ne;
        const int lb = le < EPB ? le : 0;
        const T* sx = stage + s * (SX + SO) + lb * ND;
        const T* so = stage + s * (SX + SO) + SX + lb * NQ;
        mass_element<T, int>(sx, so, y + (active ? e : 0) * ND, b, bufs + (2 * lb) * MD, bufs + (2 * lb + 1) * MD,
                             DIM, D, Q, M, r % M, r / M, active);
        __syncthreads();   // stage s is read: the next iteration's copies may overwrite it
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// 2-D, one thread per element (tile {EPB, 2, 0, 0}): the same four
// contractions and the scaling, every value in the thread's registers and
// no barrier after B1 is staged.  The x stage T1[jy][qx] = sum_jx
// B1[qx][jx] X[jy][jx] is kept whole (D x Q); the rest goes one quadrature
// row qy at a time: T2[qx] = op[qy][qx] sum_jy B1[qy][jy] T1[jy][qx],
// T3[jx] = sum_qx B1[qx][jx] T2[qx], and Y[jy][jx] += B1[qy][jy] T3[jx].
// Each thread reads its element's x and op rows through L1 (a warp's
// elements are contiguous, so every line it touches is used whole).
template <class T, int D, int Q, int EPB>
__global__ void __launch_bounds__(cjg::mass_threads(D, Q, EPB, 2))
mass_apply_thread(const T* __restrict__ B1, const T* __restrict__ op, const T* __restrict__ x, T* __restrict__ y,
                  long long ne) {
    static_assert(cjg::mass_thread_ok(2, D, Q), "one thread per element keeps D Q + D^2 <= 80 values");
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* b = reinterpret_cast<T*>(cj_smem);   // B1, Q x D (cjg::mass_smem, form 2)
    for (int i = threadIdx.x; i < Q * D; i += blockDim.x) b[i] = B1[i];
    __syncthreads();
    const long long e = (long long)blockIdx.x * EPB + threadIdx.x;
    if (threadIdx.x >= EPB || e >= ne) return;
    const T* xe = x + e * (D * D);
    const T* oe = op + e * (Q * Q);
    T t1[D][Q];
#pragma unroll
    for (int jy = 0; jy < D; ++jy) {
        T xr[D];
#pragma unroll
        for (int jx = 0; jx < D; ++jx) xr[jx] = __ldg(xe + jy * D + jx);
#pragma unroll
        for (int qx = 0; qx < Q; ++qx) {
            T s = T(0);
#pragma unroll
            for (int jx = 0; jx < D; ++jx) s = mass_fma(b[qx * D + jx], xr[jx], s);
            t1[jy][qx] = s;
        }
    }
    T yv[D][D];
#pragma unroll
    for (int jy = 0; jy < D; ++jy)
#pragma unroll
        for (int jx = 0; jx < D; ++jx) yv[jy][jx] = T(0);
#pragma unroll
    for (int qy = 0; qy < Q; ++qy) {
        T t2[Q];
#pragma unroll
        for (int qx = 0; qx < Q; ++qx) {
            T s = T(0);
#pragma unroll
            for (int jy = 0; jy < D; ++jy) s = mass_fma(b[qy * D + jy], t1[jy][qx], s);
            t2[qx] = __ldg(oe + qy * Q + qx) * s;
        }
#pragma unroll
        for (int jx = 0; jx < D; ++jx) {
            T s = T(0);
#pragma unroll
            for (int qx = 0; qx < Q; ++qx) s = mass_fma(b[qx * D + jx], t2[qx], s);
#pragma unroll
            for (int jy = 0; jy < D; ++jy) yv[jy][jx] = mass_fma(b[qy * D + jy], s, yv[jy][jx]);
        }
    }
    T* ye = y + e * (D * D);
#pragma unroll
    for (int jy = 0; jy < D; ++jy)
#pragma unroll
        for (int jx = 0; jx < D; ++jx) ye[jy * D + jx] = yv[jy][jx];
}

// Generic: run-time dimension, D, Q and elements per block (the same stages
// with run-time loop bounds).
template <class T>
__global__ void __launch_bounds__(1024)
mass_apply_generic(const T* __restrict__ B1, const T* __restrict__ op, const T* __restrict__ x, T* __restrict__ y,
                   long long ne, int dim, int D, int Q, int epb) {
    const int M = D > Q ? D : Q;
    const int ND = dim == 2 ? D * D : D * D * D, NQ = dim == 2 ? Q * Q : Q * Q * Q;
    const int MD = dim == 2 ? M * M : M * M * M;
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* b = reinterpret_cast<T*>(cj_smem);
    T* bufs = b + cjg::mass_b_elems(D, Q);
    const int t = threadIdx.x, le = t / (M * M), r = t - le * M * M;
    for (int i = t; i < Q * D; i += blockDim.x) b[i] = B1[i];
    const long long e = (long long)blockIdx.x * epb + le;
    const bool active = le < epb && e < ne;
    const long long ec = active ? e : 0;
    const int lb = le < epb ? le : 0;
    mass_element<T, int>(x + ec * ND, op + ec * NQ, y + ec * ND, b, bufs + (2 * lb) * MD, bufs + (2 * lb + 1) * MD,
                         dim, D, Q, M, r % M, r / M, active);
}

}  // namespace cj
#endif
