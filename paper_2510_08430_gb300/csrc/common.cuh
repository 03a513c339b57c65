// Shared device helpers for the block-layer SR kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include "../../include/nqs_sr.h"

namespace nqs {

// ---------------------------------------------------------------- complex
template <typename R> struct alignas(2 * sizeof(R)) cx { R re, im; };
using c64 = cx<float>;
using c128 = cx<double>;

template <typename R> __host__ __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> z; z.re = a; z.im = b; return z; }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> __host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk<R>(s * a.re, s * a.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> cconj(cx<R> a) { return mk<R>(a.re, -a.im); }
template <typename R> __host__ __device__ __forceinline__ R cabs2(cx<R> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <typename R> __host__ __device__ __forceinline__ void cmac(cx<R>& acc, cx<R> a, cx<R> b) {
    acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
    acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <typename R> __host__ __device__ __forceinline__ void cmacc(cx<R>& acc, cx<R> a, cx<R> b) {
    acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
    acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
template <typename To, typename Ti> __host__ __device__ __forceinline__ cx<To> ccast(cx<Ti> a) {
    return mk<To>((To)a.re, (To)a.im);
}

__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }

// complex exp
template <typename R> __device__ __forceinline__ cx<R> cexp_(cx<R> z) {
    R s, c;
    sincos_(z.im, &s, &c);
    R m = exp(z.re);
    return mk<R>(m * c, m * s);
}

// ln cosh with the branch s z - ln2 + log1p(exp(-2 s z)), s = sign(Re z) (+1 at 0).
// With u = exp(-2 s z) = rho e^{i t}, rho = exp(-2|x|) <= 1, t = -2 s y:
//   |1 + u|^2 = (1 - rho)^2 + 4 rho cos^2(t/2)   (a sum of non-negative terms),
//   log1p(u) = 0.5 log|1 + u|^2 + i atan2(rho sin t, (1 - rho) + 2 rho cos^2(t/2)).
// The modulus uses log1p(2 rho cos t + rho^2) when |1+u|^2 is not small and the
// cancellation-free sum otherwise (near the zeros of cosh).
template <typename R> __device__ __forceinline__ cx<R> clncosh(cx<R> z) {
    const R s = (z.re >= R(0)) ? R(1) : R(-1);
    const R ax = s * z.re;                 // >= 0
    const R h = -s * z.im;                 // t / 2
    R sh, ch;
    sincos_(h, &sh, &ch);
    const R rho = exp(R(-2) * ax);
    const R om = -expm1(R(-2) * ax);       // 1 - rho
    const R c2 = ch * ch;
    const R mod2 = fma(om, om, R(4) * rho * c2);
    const R cost = fma(R(2), c2, R(-1));   // cos t
    const R sint = R(2) * sh * ch;         // sin t
    const R lr = (mod2 > R(0.5)) ? R(0.5) * log1p(fma(R(2) * rho, cost, rho * rho)) : R(0.5) * log(mod2);
    const R li = atan2(rho * sint, fma(R(2) * rho, c2, om));
    return mk<R>(ax - R(0.6931471805599453094172321) + lr, s * z.im + li);
}

// tanh(z) for x = Re z >= 0 from q = exp(-2z) = rho (cos 2y - i sin 2y), rho = exp(-2x):
//   tanh z = (1 - q)/(1 + q) = ((1 - rho^2) + 2 i rho sin 2y) / |1 + q|^2,
//   |1 + q|^2 = (1 - rho)^2 + 4 rho cos^2 y   (no cancellation near the poles),
// 1 - rho^2 = (1 - rho)(1 + rho) with 1 - rho = -expm1(-2x); odd symmetry for x < 0.
template <typename R> __device__ __forceinline__ cx<R> ctanh(cx<R> z) {
    const R s = (z.re >= R(0)) ? R(1) : R(-1);
    const R x = s * z.re, y = s * z.im;  // x >= 0
    R sy, cy;
    sincos_(y, &sy, &cy);
    const R rho = exp(R(-2) * x);
    const R om = -expm1(R(-2) * x);
    const R d = fma(om, om, R(4) * rho * cy * cy);
    const R re = om * (R(1) + rho) / d;
    const R im = R(4) * rho * sy * cy / d;
    return mk<R>(s * re, s * im);
}

// ---------------------------------------------------------------- reductions
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename R> __device__ __forceinline__ cx<R> warp_sum(cx<R> v) {
    v.re = warp_sum(v.re);
    v.im = warp_sum(v.im);
    return v;
}
// Block-wide sum; `sh` holds >= 32 entries of T; all threads receive the result.
template <typename T> __device__ __forceinline__ T block_sum(T v, T* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- device status
// First 256 bytes of every workspace. The first non-zero code wins.
struct DevStatus {
    int code;
    int where;
    long long detail;
};
__device__ __forceinline__ void set_status(DevStatus* st, int code, int where, long long detail) {
    if (st == nullptr) return;
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->where = where;
        st->detail = detail;
    }
}
template <typename R> __device__ __forceinline__ bool finite_cx(cx<R> z) { return isfinite(z.re) && isfinite(z.im); }

// where-codes for DevStatus (identify the kernel that reported)
enum : int {
    W_JAC = 1, W_ELOC = 2, W_CENTER = 3, W_GRAM = 4, W_GRAM_TC = 5, W_TRD = 6, W_BISECT = 7,
    W_SOLVE = 8, W_QL = 9,
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Host-side count of kernel launches issued by this library (all threads).
unsigned long long& launch_counter();
inline void count_launch() { __atomic_add_fetch(&launch_counter(), 1ull, __ATOMIC_RELAXED); }

}  // namespace nqs
