// tt_internal.cuh -- device building blocks shared by the TT kernels.
//
// Tall-skinny QR on one GPU (the TSQR idea of Sec. 3.3, mapped onto CTAs):
//   * a "leaf" CTA owns a contiguous range of mode slices of one core and runs a
//     sequential (flat-tree) Householder QR over tiles of those slices: each tile is
//     stacked under the CTA's running triangular factor and factored;
//   * a G-ary tree of "node" CTAs then factors the stacked leaf triangles in the
//     same way, level by level (one launch per level);
//   * the orthogonal factor stays implicit (Sec. 3.5): tile and node reflectors are
//     stored, and Q [C; 0] is applied later from the root down (TSQR-Apply-Q,
//     Alg. 4), again as a sequence of stacked-tile reflections.
// All of it reduces to two block-level routines on a stacked matrix
// [Rr (k rows); tile (M rows)] with b columns: hh_factor and hh_apply.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace ttgb {

constexpr int NT = 256;  // threads per CTA of every bulk kernel

// ------------------------------------------------------------------------------------
// df32: a value stored as an unevaluated sum hi + lo of two FP32 numbers ("double-word"
// or double-single arithmetic).  Built from the error-free transformations TwoSum
// (Knuth), FastTwoSum (Dekker) and the FMA-based exact product, in the forms analysed by
// Joldes, Muller, Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic" (ACM TOMS 2017): addition (their accurate DW+DW), multiplication
// (DW x DW with FMA), division and square root by one correction step.  Relative accuracy
// about 2^-46, computed entirely on the FP32 pipes (58x the FP64 rate on GB300).
// ------------------------------------------------------------------------------------

struct df32 {
  float hi, lo;
  __host__ __device__ df32() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df32(float x) : hi(x), lo(0.f) {}
  __host__ __device__ df32(int x) : hi((float)x), lo(0.f) {}
  __device__ explicit df32(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ df32 operator+(df32 x, df32 y) {
  float s, e, t, f;
  two_sum(x.hi, y.hi, s, e);
  two_sum(x.lo, y.lo, t, f);
  e += t;
  fast_two_sum(s, e, s, e);
  e += f;
  fast_two_sum(s, e, s, e);
  return df32(s, e);
}
__device__ __forceinline__ df32 operator-(df32 x) { return df32(-x.hi, -x.lo); }
__device__ __forceinline__ df32 operator-(df32 x, df32 y) { return x + (-y); }
__device__ __forceinline__ df32 operator*(df32 x, df32 y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float s;
  fast_two_sum(p, e, s, e);
  return df32(s, e);
}
__device__ __forceinline__ df32 operator/(df32 x, df32 y) {
  const float q = x.hi / y.hi;
  const df32 r = x - df32(q) * y;  // remainder, nearly exact
  const float q2 = r.hi / y.hi;
  float s, e;
  fast_two_sum(q, q2, s, e);
  return df32(s, e);
}
__device__ __forceinline__ df32 &operator+=(df32 &x, df32 y) { return x = x + y; }
__device__ __forceinline__ df32 &operator-=(df32 &x, df32 y) { return x = x - y; }
__device__ __forceinline__ df32 &operator*=(df32 &x, df32 y) { return x = x * y; }
__device__ __forceinline__ bool operator==(df32 x, df32 y) { return x.hi == y.hi && x.lo == y.lo; }
__device__ __forceinline__ bool operator!=(df32 x, df32 y) { return !(x == y); }
__device__ __forceinline__ bool operator>=(df32 x, df32 y) {
  return x.hi > y.hi || (x.hi == y.hi && x.lo >= y.lo);
}
__device__ __forceinline__ df32 df_sqrt(df32 x) {
  if (x.hi <= 0.f) return df32(0.f);
  const float sq = sqrtf(x.hi);
  // x - sq^2 with the exact product sq * sq
  const float p = sq * sq;
  const float pe = fmaf(sq, sq, -p);
  const df32 r = x - df32(p, pe);
  const float c = r.hi / (2.f * sq);
  float s, e;
  fast_two_sum(sq, c, s, e);
  return df32(s, e);
}

// accumulate a + b * c into an unevaluated (s, comp) pair: the compensated dot product
// of Ogita, Rump, Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005,
// Dot2) extended to double-word operands; finish with df_finish(s, comp).
__device__ __forceinline__ void df_dot_acc(float &s, float &comp, df32 b, df32 c) {
  const float p = b.hi * c.hi;
  float e = fmaf(b.hi, c.hi, -p);
  e = fmaf(b.hi, c.lo, e);
  e = fmaf(b.lo, c.hi, e);
  float t;
  two_sum(s, p, s, t);
  comp += t + e;
}
__device__ __forceinline__ df32 df_finish(float s, float comp) {
  float h, l;
  fast_two_sum(s, comp, h, l);
  return df32(h, l);
}
// x - v * w with one normalisation
__device__ __forceinline__ df32 df_sub_prod(df32 x, df32 v, df32 w) {
  const float p = v.hi * w.hi;
  float e = fmaf(v.hi, w.hi, -p);
  e = fmaf(v.hi, w.lo, e);
  e = fmaf(v.lo, w.hi, e);
  float s, t;
  two_sum(x.hi, -p, s, t);
  t += x.lo - e;
  fast_two_sum(s, t, s, t);
  return df32(s, t);
}

template <typename T>
struct is_df : std::false_type {};
template <>
struct is_df<df32> : std::true_type {};

template <typename T>
__device__ __forceinline__ T tsqrt(T x);
template <>
__device__ __forceinline__ double tsqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float tsqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ df32 tsqrt<df32>(df32 x) { return df_sqrt(x); }

// FP64 reciprocal and reciprocal square root by Newton-Raphson iteration from a
// single-precision hardware seed.  On GB300 every FP64 instruction occupies an SMSP's
// FP64 unit for about 64 cycles and the FP64 divide / square root sequences take about
// 650-700 cycles; these take about 8 FP64 instructions.  The argument is first scaled by
// a power of two (exponent arithmetic on the bit pattern) into [1, 2) resp. [1, 4) so the
// seed never under- or overflows; two Newton steps take the seed's ~2^-22 relative error
// below FP64 rounding.  Valid for finite, normal, nonzero x (x > 0 for rsqrt_nr).
__device__ __forceinline__ double rcp_nr(double x) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff) - 1023;
  const double m = __longlong_as_double(bits - ((long long)ex << 52));  // |m| in [1, 2)
  double y = (double)__frcp_rn((float)m);
  // y <- y (2 - m y), written as y + y (1 - m y)
  double e = fma(-m, y, 1.0);
  y = fma(y, e, y);
  e = fma(-m, y, 1.0);
  y = fma(y, e, y);
  return __longlong_as_double(__double_as_longlong(y) - ((long long)ex << 52));
}

__device__ __forceinline__ double rsqrt_nr(double x) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff) - 1023;
  const int k = ex >> 1;  // floor(ex / 2)
  const double m = __longlong_as_double(bits - ((long long)(2 * k) << 52));  // in [1, 4)
  double y = (double)rsqrtf((float)m);
  const double hm = 0.5 * m;
  // y <- y (3 - m y^2) / 2
  y = y * fma(-hm, y * y, 1.5);
  y = y * fma(-hm, y * y, 1.5);
  return __longlong_as_double(__double_as_longlong(y) - ((long long)k << 52));
}

// x in the range where the Newton helpers apply (normal, far from overflow)
__device__ __forceinline__ bool nr_range(double x) { return x > 1e-290 && x < 1e290; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <>
__device__ __forceinline__ df32 warp_sum<df32>(df32 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df32 u(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    v = v + u;
  }
  return v;
}

// ------------------------------------------------------------------------------------
// exponent range of carried factors
// ------------------------------------------------------------------------------------
// A TT's norm is a product of N per-core factors, so the small matrices carried from core
// to core (the pushed R of the orthogonalization, the partial contraction W of the inner
// product) can drift by a fixed factor per core: a Hadamard product of two unit-norm TTs
// with 30 modes of size 1024 has norm near 2^-150, out of FP32 range.  Carried factors are
// therefore kept in [2^-32, 2^32] by exact power-of-two rescaling, and the exponent is
// accumulated separately.

// Largest |v[i]| over the block (any block size that is a multiple of 32, up to 1024).
__device__ __forceinline__ double block_absmax(const double *v, int n, double *red32) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red32[threadIdx.x >> 5] = m;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red32[w]);
  __syncthreads();
  return r;
}

// Power-of-two exponent to divide out of a factor whose largest entry is m: zero while m
// stays in [2^-32, 2^32] (and for a zero or non-finite factor), else the binary exponent of m.
__device__ __forceinline__ int range_exp(double m) {
  if (!(m > 0.0) || !isfinite(m) || (m >= 0x1p-32 && m <= 0x1p32)) return 0;
  return ilogb(m);
}

// Scratch a block-level routine needs in shared memory.
template <typename T>
struct Scratch {
  T *red;   // NT elements
  T *wbuf;  // >= max columns elements (NT for hh_apply_grouped)
  T *sc;    // 4 elements (two reflectors' scale and tau)
};

// H = I - tau u u^T with u = [1; v], v_r = V[r * ldv] for r in [r0, M), applied to the
// stacked matrix [p (nc entries); X rows r0..M-1 (nc entries each, row stride ldx)].
// Thread t owns column c = t mod nc of row group g = t / nc (G = NT / nc groups, so short
// trailing blocks still spread over the whole CTA); the partial dot products are summed by
// a tree in shared memory, then w_c = tau (p_c + v^T X(:, c)) and X -= v w^T over the dense
// block.  All threads of the CTA must call it with identical arguments; nc <= NT.
// vscale: v = vscale * V (a reflector whose scaling is still pending); w and the update
// are formed from the unscaled V.
template <typename T>
__device__ void reflect(T tau, const T *V, int ldv, int r0, int M, T *p, T *X, int ldx, int nc, Scratch<T> s,
                        T vscale = T(1)) {
  if (nc <= 0) return;
  const int t = threadIdx.x;
  const int nrow = M - r0;
  int G = NT / nc;
  if (G > nrow) G = nrow > 0 ? nrow : 1;
  if (t < G * nc) {
    const int g = t / nc, c = t - g * nc;
    if constexpr (is_df<T>::value) {
      float sh = 0.f, sl = 0.f;
      for (int r = r0 + g; r < M; r += G) df_dot_acc(sh, sl, V[(size_t)r * ldv], X[(size_t)r * ldx + c]);
      s.red[g * nc + c] = df_finish(sh, sl);
    } else {
      T acc = T(0);
      for (int r = r0 + g; r < M; r += G) acc += V[(size_t)r * ldv] * X[(size_t)r * ldx + c];
      s.red[g * nc + c] = acc;
    }
  }
  __syncthreads();
  for (int h = G; h > 1;) {
    const int half = (h + 1) >> 1;
    for (int idx = t; idx < (h - half) * nc; idx += NT) s.red[idx] += s.red[idx + half * nc];
    h = half;
    __syncthreads();
  }
  if (t < nc) {
    const T w = tau * (p[t] + vscale * s.red[t]);
    s.wbuf[t] = vscale * w;
    p[t] -= w;
  }
  __syncthreads();
  if (nrow > 0) {
    // dense walk over the nrow x nc block without per-element division
    const int dq = NT / nc, dr = NT - dq * nc;
    int r = t / nc, cc = t - (t / nc) * nc;
    for (; r < nrow;) {
      const size_t rr = (size_t)(r0 + r);
      if constexpr (is_df<T>::value) {
        T &x = X[rr * ldx + cc];
        x = df_sub_prod(x, V[rr * ldv], s.wbuf[cc]);
      } else {
        X[rr * ldx + cc] -= V[rr * ldv] * s.wbuf[cc];
      }
      r += dq;
      cc += dr;
      if (cc >= nc) {
        cc -= nc;
        ++r;
      }
    }
  }
  __syncthreads();
}

// Householder QR step of the stacked matrix [Rr rows 0..k-1; tile rows 0..M-1], b columns,
// LAPACK conventions (H_j = I - tau_j u u^T, u_pivot = 1, beta = -sign(alpha) ||x||,
// tau = 0 when the part below the pivot is zero).  Reflector j pivots on Rr row j when
// j < k, otherwise on tile row j-k; kk = min(k + M, b) reflectors.  On return Rr rows
// 0..k-1 hold updated R rows; tile entries (r, c) with c < k + r hold reflector entries
// and, for r < kk - k, entries c >= k + r hold R row k + r.  tau[0..kk-1] is written.
// Rr and tile are row-major with leading dimensions ldr, ldt.  Returns kk.
// tri_off >= 0 declares the tile as q upper-triangular factors interleaved row by row
// (tile row r q + i is row r of factor i, starting at column r + tri_off): reflector j then
// only touches tile rows < (j - tri_off + 1) q, the others being zero in column j.  q = 1
// is a single triangle stacked under Rr.  tri_off < 0: dense tile.
__device__ __forceinline__ int tile_rows_for(int j, int M, int tri_off, int q = 1) {
  return tri_off < 0 ? M : min(M, max(0, (j - tri_off + 1) * q));
}

// Reflector-by-reflector forms, used for the FP32-storage compute types (df32, float), whose
// serial chains are short on the wide FP32 pipes.
template <typename T>
__device__ int hh_factor_seq(T *Rr, int ldr, int k, T *tile, int ldt, int M, int b, T *tau, Scratch<T> s,
                         int tri_off = -1, int q = 1) {
  const int kk = min(k + M, b);
  // Narrow factors: warp 0 forms reflector j (column norm, square root, reciprocal) while
  // the other warps apply the scaling still owed by the stored column of reflector pj
  // (rows pr0..pM-1); then the whole CTA applies reflector j.
  int pj = -1, pr0 = 0, pM = 0;
  T pend = T(1);
  for (int j = 0; j < kk; ++j) {
    const int r0 = j < k ? 0 : j - k + 1;
    const int Mj = tile_rows_for(j, M, tri_off, q);
    T *piv = j < k ? Rr + (size_t)j * ldr : tile + (size_t)(j - k) * ldt;
    if (threadIdx.x >= 32 && pj >= 0) {
      for (int r = pr0 + (int)threadIdx.x - 32; r < pM; r += NT - 32) tile[(size_t)r * ldt + pj] *= pend;
    }
    if (threadIdx.x < 32) {
      T ss = T(0);
      for (int r = r0 + threadIdx.x; r < Mj; r += 32) {
        const T v = tile[(size_t)r * ldt + j];
        ss += v * v;
      }
      ss = warp_sum(ss);
      if (threadIdx.x == 0) {
        T tj = T(0), scale = T(0);
        if (ss != T(0)) {
          const T alpha = piv[j];
          const T v = alpha * alpha + ss;
          const bool fast = std::is_same<T, double>::value && nr_range((double)v);
          const T nrm = fast ? (T)((double)v * rsqrt_nr((double)v)) : tsqrt(v);
          const T beta = alpha >= T(0) ? -nrm : nrm;
          const T d = alpha - beta;
          const T bd = beta * d;
          if (fast && nr_range(fabs((double)bd))) {
            // one reciprocal: with q = 1 / (beta d), tau = (beta - alpha) / beta = -d d q
            // and 1 / d = beta q
            const T q = (T)rcp_nr((double)bd);
            tj = -d * d * q;
            scale = beta * q;
          } else {
            // textbook form; tau lies in [1, 2] whatever the scale of the column
            tj = (beta - alpha) / beta;
            scale = T(1) / d;
          }
          piv[j] = beta;
        }
        tau[j] = tj;
        s.sc[0] = scale;
        s.sc[1] = tj;
      }
    }
    __syncthreads();
    const T tj = s.sc[1];
    pj = -1;
    if (tj != T(0)) {
      const T scale = s.sc[0];
      reflect(tj, tile + j, ldt, r0, Mj, piv + j + 1, tile + j + 1, ldt, b - j - 1, s, scale);
      pj = j;
      pend = scale;
      pr0 = r0;
      pM = Mj;
    } else {
      __syncthreads();
    }
  }
  if (pj >= 0) {
    for (int r = pr0 + (int)threadIdx.x; r < pM; r += NT) tile[(size_t)r * ldt + pj] *= pend;
  }
  __syncthreads();
  return kk;
}

template <typename T>
__device__ int hh_factor_ahead(T *Rr, int ldr, int k, T *tile, int ldt, int M, int b, T *tau, Scratch<T> s,
                         int tri_off = -1, int q = 1) {
  const int kk = min(k + M, b);
  const int t = threadIdx.x;
  // Wide factors: warp 0 forms reflector j (column norm, then the square root / reciprocal
  // chain) while the other warps apply the scaling still owed by the stored column of
  // reflector pj (rows pr0..pM-1) and already take the dot products of reflector j's
  // unscaled column with the trailing columns (the scalars are needed only when w is
  // formed).
  const int nth = NT - 32;
  int pj = -1, pr0 = 0, pM = 0;
  T pend = T(1);
  auto dots = [&](int u, int j, int r0, int Mj, int nc, int G) {
    if (nc > 0 && u < G * nc) {
      const int g = u / nc, c = u - g * nc;
      const T *X = tile + j + 1 + c;
      if constexpr (is_df<T>::value) {
        float sh = 0.f, sl = 0.f;
        for (int r = r0 + g; r < Mj; r += G) df_dot_acc(sh, sl, tile[(size_t)r * ldt + j], X[(size_t)r * ldt]);
        s.red[g * nc + c] = df_finish(sh, sl);
      } else {
        T acc = T(0);
        for (int r = r0 + g; r < Mj; r += G) acc += tile[(size_t)r * ldt + j] * X[(size_t)r * ldt];
        s.red[g * nc + c] = acc;
      }
    }
  };
  for (int j = 0; j < kk; ++j) {
    const int r0 = j < k ? 0 : j - k + 1;
    const int Mj = tile_rows_for(j, M, tri_off, q);
    T *piv = j < k ? Rr + (size_t)j * ldr : tile + (size_t)(j - k) * ldt;
    const int nc = b - j - 1, nrow = Mj - r0;
    // dot-product groups over the nth threads taking them (nc < b <= TT_MAX_RANK < NT - 32)
    int G = nc > 0 ? nth / nc : 1;
    if (G > nrow) G = nrow > 0 ? nrow : 1;
    if (t < 32) {
      T ss = T(0);
      for (int r = r0 + t; r < Mj; r += 32) {
        const T v = tile[(size_t)r * ldt + j];
        ss += v * v;
      }
      ss = warp_sum(ss);
      if (t == 0) {
        T tj = T(0), scale = T(0);
        if (ss != T(0)) {
          const T alpha = piv[j];
          const T v = alpha * alpha + ss;
          const bool fast = std::is_same<T, double>::value && nr_range((double)v);
          const T nrm = fast ? (T)((double)v * rsqrt_nr((double)v)) : tsqrt(v);
          const T beta = alpha >= T(0) ? -nrm : nrm;
          const T d = alpha - beta;
          const T bd = beta * d;
          if (fast && nr_range(fabs((double)bd))) {
            // one reciprocal: with q = 1 / (beta d), tau = (beta - alpha) / beta = -d d q
            // and 1 / d = beta q
            const T qq = (T)rcp_nr((double)bd);
            tj = -d * d * qq;
            scale = beta * qq;
          } else {
            // textbook form; tau lies in [1, 2] whatever the scale of the column
            tj = (beta - alpha) / beta;
            scale = T(1) / d;
          }
          piv[j] = beta;
        }
        tau[j] = tj;
        s.sc[0] = scale;
        s.sc[1] = tj;
      }
    } else {
      const int u = t - 32;
      if (pj >= 0)
        for (int r = pr0 + u; r < pM; r += NT - 32) tile[(size_t)r * ldt + pj] *= pend;
      dots(u, j, r0, Mj, nc, G);
    }
    __syncthreads();
    const T tj = s.sc[1];
    pj = -1;
    if (tj != T(0)) {
      const T scale = s.sc[0];
      if (nc > 0) {
        for (int h = G; h > 1;) {
          const int half = (h + 1) >> 1;
          for (int idx = t; idx < (h - half) * nc; idx += NT) s.red[idx] += s.red[idx + half * nc];
          h = half;
          __syncthreads();
        }
        T *p = piv + j + 1;
        if (t < nc) {
          const T w = tj * (p[t] + scale * s.red[t]);
          s.wbuf[t] = scale * w;
          p[t] -= w;
        }
        __syncthreads();
        if (nrow > 0) {
          // dense walk over the nrow x nc trailing block: X -= v w^T (v unscaled, w scaled)
          const int dq = NT / nc, dr = NT - dq * nc;
          int r = t / nc, cc = t - (t / nc) * nc;
          for (; r < nrow;) {
            const size_t rr = (size_t)(r0 + r);
            if constexpr (is_df<T>::value) {
              T &x = tile[rr * ldt + j + 1 + cc];
              x = df_sub_prod(x, tile[rr * ldt + j], s.wbuf[cc]);
            } else {
              tile[rr * ldt + j + 1 + cc] -= tile[rr * ldt + j] * s.wbuf[cc];
            }
            r += dq;
            cc += dr;
            if (cc >= nc) {
              cc -= nc;
              ++r;
            }
          }
        }
      }
      pj = j;
      pend = scale;
      pr0 = r0;
      pM = Mj;
    }
    __syncthreads();
  }
  if (pj >= 0) {
    for (int r = pr0 + t; r < pM; r += NT) tile[(size_t)r * ldt + pj] *= pend;
  }
  __syncthreads();
  return kk;
}

// Named CTA barriers (PTX bar.sync / bar.arrive with an id and a thread count; id 0 is
// __syncthreads).  bar.arrive lets a warp signal a barrier without waiting at it.
__device__ __forceinline__ void nbar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Scalars of one Householder reflector (LAPACK convention): from the pivot alpha and the
// sum of squares ss of the entries below it, beta = -sign(alpha) sqrt(alpha^2 + ss),
// tau = (beta - alpha) / beta and the scale 1 / (alpha - beta) of the stored column;
// tau = 0 (identity) when ss = 0.
template <typename T>
__device__ __forceinline__ void house_scalars(T alpha, T ss, T &tj, T &scale, T &beta) {
  tj = T(0);
  scale = T(0);
  beta = alpha;
  if (ss == T(0)) return;
  const T v = alpha * alpha + ss;
  const bool fast = std::is_same<T, double>::value && nr_range((double)v);
  const T nrm = fast ? (T)((double)v * rsqrt_nr((double)v)) : tsqrt(v);
  beta = alpha >= T(0) ? -nrm : nrm;
  const T d = alpha - beta;
  const T bd = beta * d;
  if (fast && nr_range(fabs((double)bd))) {
    // one reciprocal: with q = 1 / (beta d), tau = (beta - alpha) / beta = -d d q and 1 / d = beta q
    const T qq = (T)rcp_nr((double)bd);
    tj = -d * d * qq;
    scale = beta * qq;
  } else {
    // textbook form; tau lies in [1, 2] whatever the scale of the column
    tj = (beta - alpha) / beta;
    scale = T(1) / d;
  }
}

// Householder QR of the stacked matrix with look-ahead (layout and conventions as described
// above).  Warp 0 forms the reflectors: while warps 1..7 take the dot products of
// reflector j with the trailing columns and apply it to columns j+2.., warp 0 applies it
// to column j+1 first, then computes the norm and the scalar chain (square root,
// reciprocal) of reflector j+1, so that the ~30 dependent FP64 instructions of each chain
// (each holding an SMSP's FP64 unit ~64 cycles on GB300) run beside the bulk work instead
// of before it.  Named barriers: 1 among warps 1..7 (their reduction), 2 "scalars of the
// next reflector ready" (warp 0 arrives), 3 "w ready" (all wait), 4 "column j+1 and all
// updates done" (warp 0 arrives).  The stored column of reflector j is scaled by its
// 1 / (alpha - beta) one step later, when nothing reads it any more.
template <typename T>
__device__ int hh_factor_la(T *Rr, int ldr, int k, T *tile, int ldt, int M, int b, T *tau, Scratch<T> s,
                            int tri_off = -1, int q = 1) {
  constexpr int NB = NT - 32;  // threads of warps 1..7
  const int kk = min(k + M, b);
  const int t = threadIdx.x;
  const bool cw = t < 32;
  const int u = t - 32;
  auto pivrow = [&](int j) -> T * { return j < k ? Rr + (size_t)j * ldr : tile + (size_t)(j - k) * ldt; };
  auto rows0 = [&](int j) { return j < k ? 0 : j - k + 1; };
  // warp 0: scalars of reflector j from its (updated) column, published in slot j & 1
  auto form = [&](int j) {
    const int r0 = rows0(j), Mj = tile_rows_for(j, M, tri_off, q);
    T ss = T(0);
    for (int r = r0 + t; r < Mj; r += 32) {
      const T v = tile[(size_t)r * ldt + j];
      ss += v * v;
    }
    ss = warp_sum(ss);
    if (t == 0) {
      T *piv = pivrow(j);
      T tj, scale, beta;
      house_scalars(piv[j], ss, tj, scale, beta);
      piv[j] = beta;
      tau[j] = tj;
      s.sc[2 * (j & 1)] = scale;
      s.sc[2 * (j & 1) + 1] = tj;
    }
    __syncwarp();
  };
  if (kk <= 0) {
    __syncthreads();
    return kk;
  }
  if (cw) {
    form(0);
    nbar_arrive(2, NT);
  }
  for (int j = 0; j < kk; ++j) {
    const int r0 = rows0(j), Mj = tile_rows_for(j, M, tri_off, q);
    const int nrow = Mj - r0;
    const int nc = b - j - 1;
    T *piv = pivrow(j);
    if (!cw) {
      // deferred scaling of reflector j-1's stored column (no one reads it any more)
      if (j >= 1) {
        const T sp = s.sc[2 * ((j - 1) & 1)];
        const int pr0 = rows0(j - 1), pM = tile_rows_for(j - 1, M, tri_off, q);
        for (int r = pr0 + u; r < pM; r += NB) tile[(size_t)r * ldt + j - 1] *= sp;
      }
      // dot products of the unscaled column j with the trailing columns (partials by row group)
      int G = nc > 0 ? NB / nc : 1;
      if (G > nrow) G = nrow > 0 ? nrow : 1;
      if (nc > 0 && u < G * nc) {
        const int g = u / nc, c = u - g * nc;
        const T *X = tile + j + 1 + c;
        if constexpr (is_df<T>::value) {
          float sh = 0.f, sl = 0.f;
          for (int r = r0 + g; r < Mj; r += G) df_dot_acc(sh, sl, tile[(size_t)r * ldt + j], X[(size_t)r * ldt]);
          s.red[g * nc + c] = df_finish(sh, sl);
        } else {
          T acc = T(0);
          for (int r = r0 + g; r < Mj; r += G) acc += tile[(size_t)r * ldt + j] * X[(size_t)r * ldt];
          s.red[g * nc + c] = acc;
        }
      }
      if (nc > 0) {
        nbar_sync(1, NB);
        for (int h = G; h > 1;) {
          const int half = (h + 1) >> 1;
          for (int idx = u; idx < (h - half) * nc; idx += NB) s.red[idx] += s.red[idx + half * nc];
          h = half;
          nbar_sync(1, NB);
        }
      }
      nbar_sync(2, NT);  // scalars of reflector j
      if (u < nc) {
        const T scale = s.sc[2 * (j & 1)], tj = s.sc[2 * (j & 1) + 1];
        T *p = piv + j + 1;
        const T w = tj * (p[u] + scale * s.red[u]);
        s.wbuf[u] = scale * w;
        p[u] -= w;
      }
      nbar_sync(3, NT);
      // update columns j+2.. over the reflector's rows: X -= x_j w^T (x_j unscaled, w scaled)
      const int ncu = nc - 1;
      if (ncu > 0 && nrow > 0) {
        const int dq = NB / ncu, dr = NB - dq * ncu;
        int r = u / ncu, cc = u - (u / ncu) * ncu;
        for (; r < nrow;) {
          const size_t rr = (size_t)(r0 + r);
          if constexpr (is_df<T>::value) {
            T &x = tile[rr * ldt + j + 2 + cc];
            x = df_sub_prod(x, tile[rr * ldt + j], s.wbuf[1 + cc]);
          } else {
            tile[rr * ldt + j + 2 + cc] -= tile[rr * ldt + j] * s.wbuf[1 + cc];
          }
          r += dq;
          cc += dr;
          if (cc >= ncu) {
            cc -= ncu;
            ++r;
          }
        }
      }
      nbar_sync(4, NT);
    } else {
      nbar_sync(3, NT);
      // column j+1 first
      if (nc > 0) {
        const T w1 = s.wbuf[0];
        for (int r = r0 + t; r < Mj; r += 32) {
          if constexpr (is_df<T>::value) {
            T &x = tile[(size_t)r * ldt + j + 1];
            x = df_sub_prod(x, tile[(size_t)r * ldt + j], w1);
          } else {
            tile[(size_t)r * ldt + j + 1] -= tile[(size_t)r * ldt + j] * w1;
          }
        }
      }
      __syncwarp();
      nbar_arrive(4, NT);
      if (j + 1 < kk) {
        form(j + 1);
        nbar_arrive(2, NT);
      }
    }
  }
  __syncthreads();
  // the last reflector's stored column
  {
    const int j = kk - 1;
    const T sp = s.sc[2 * (j & 1)];
    for (int r = rows0(j) + t; r < tile_rows_for(j, M, tri_off, q); r += NT) tile[(size_t)r * ldt + j] *= sp;
  }
  __syncthreads();
  return kk;
}

// Householder QR of the stacked matrix (see above): the look-ahead form.
// FP64 takes the look-ahead form: each FP64 instruction of the scalar chain holds an SMSP's
// FP64 unit ~64 cycles, so the chain must run beside the bulk work.  The FP32-storage types
// (df32, float) keep the reflector-by-reflector forms: their chains are short on the FP32
// pipes, and a single warp updating the next column and forming its reflector in double-float
// arithmetic measured slower than all warps sharing that column (N=50, I_n=16384, rank 64:
// fp32x2 2.20 s reflector by reflector, 2.50 s look-ahead).  Factors of 48 or more columns
// take reflector j's dot products while its scalars are being formed (hh_factor_ahead);
// narrower ones measured faster with all threads on the dot products after the scalars.
template <typename T>
__device__ int hh_factor(T *Rr, int ldr, int k, T *tile, int ldt, int M, int b, T *tau, Scratch<T> s,
                         int tri_off = -1, int q = 1) {
  if constexpr (std::is_same<T, double>::value) {
    return hh_factor_la(Rr, ldr, k, tile, ldt, M, b, tau, s, tri_off, q);
  } else {
    return b >= 48 ? hh_factor_ahead(Rr, ldr, k, tile, ldt, M, b, tau, s, tri_off, q)
                   : hh_factor_seq(Rr, ldr, k, tile, ldt, M, b, tau, s, tri_off, q);
  }
}

// Moves the new R rows k..kk-1 produced by hh_factor from the tile into Rr (zeroing the
// entries left of the diagonal).
template <typename T>
__device__ void hh_take_rows(T *Rr, int ldr, int k, int kk, const T *tile, int ldt, int b) {
  const int n = (kk - k) * b;
  for (int idx = threadIdx.x; idx < n; idx += NT) {
    const int r = idx / b, c = idx - r * b;
    Rr[(size_t)(k + r) * ldr + c] = c >= k + r ? tile[(size_t)r * ldt + c] : T(0);
  }
  __syncthreads();
}

// Applies the orthogonal factor of one hh_factor step, Q_t = H_0 ... H_{kk-1}, to the
// stacked block [CR (k rows); CT (M rows)] of nc columns (row-major, leading dims ldcr,
// ldct): reflectors are applied from kk-1 down to 0.  V / tau are the stored tile and
// tau of that step (V row-major, ld ldv); tri_off as in hh_factor.
template <typename T>
__device__ void hh_apply(const T *V, int ldv, const T *tau, int k, int M, int b, T *CR, int ldcr, T *CT, int ldct,
                         int nc, Scratch<T> s, int tri_off = -1, int q = 1) {
  const int kk = min(k + M, b);
  for (int j = kk - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj == T(0)) continue;
    const int r0 = j < k ? 0 : j - k + 1;
    T *piv = j < k ? CR + (size_t)j * ldcr : CT + (size_t)(j - k) * ldct;
    reflect(tj, V + j, ldv, r0, tile_rows_for(j, M, tri_off, q), piv, CT, ldct, nc, s);
  }
}

// ------------------------------------------------------------------------------------
// Grouped application of one dense tile's reflectors (compact WY form)
// ------------------------------------------------------------------------------------
// The product of g consecutive reflectors H_{j0} ... H_{j0+g-1} is I - U T U^T with
// U = [u_{j0} .. u_{j0+g-1}] and T upper triangular: T_ii = tau_i,
// T(0:i, i) = -tau_i T(0:i, 0:i) U(:, 0:i)^T u_i (the forward accumulation of Schreiber
// and Van Loan, "A storage-efficient WY representation for products of Householder
// transformations", SIAM J. Sci. Stat. Comput. 1989).  Applying the group is then
// C <- C - U (T (U^T C)): one set of dot products, one reduction and one update per g
// reflectors instead of per reflector, which removes most of the CTA barriers and the
// partial-warp reductions that leave the FP64 pipe idle in the reflector-by-reflector
// form.  Reflector j of the tile has its unit pivot in CR row j (j < k) or tile row
// j - k, and stored entries V(r, j) on tile rows r > j - k (all rows when j < k).

// group size for C blocks of nc columns: g * nc dot products must fit the CTA
__device__ __host__ __forceinline__ int apply_group(int nc) {
  const int g = nc > 0 ? NT / nc : 4;
  return g >= 4 ? 4 : (g < 1 ? 1 : g);
}
// entries of the per-tile T storage (packed upper triangles of 10 entries, one per group) for
// b reflectors applied to blocks of at most nc columns
__device__ __host__ __forceinline__ int apply_tstore(int b, int nc) {
  const int g = apply_group(nc);
  return ((b + g - 1) / g) * 10 + 10;
}

template <typename T>
__device__ __forceinline__ T refl_entry(const T *V, int ldv, int k, int j, int r) {
  if (j < k) return V[(size_t)r * ldv + j];
  const int pr = j - k;
  return r > pr ? V[(size_t)r * ldv + j] : (r == pr ? T(1) : T(0));
}

// index of T(a, b) (a <= b < 4) in a group's packed upper triangle
__device__ __forceinline__ int tri_idx(int a, int b) { return a + (b * (b + 1)) / 2; }

// Q_t [CR; CT] for the reflectors of one hh_factor step on a dense tile (see hh_apply);
// Tst: scratch of apply_tstore(b, nc) elements; s.wbuf must hold NT elements.
template <typename T>
__device__ void hh_apply_grouped(const T *V, int ldv, const T *tau, int k, int M, int b, T *CR, int ldcr, T *CT,
                                 int ldct, int nc, Scratch<T> s, T *Tst) {
  if constexpr (!std::is_same<T, double>::value) {
    // FP32-storage types: reflector by reflector (their reductions are cheap on the FP32
    // pipes; the grouped form measured slower there)
    hh_apply(V, ldv, tau, k, M, b, CR, ldcr, CT, ldct, nc, s);
    return;
  }
  const int kk = min(k + M, b);
  if (kk <= 0 || nc <= 0) return;
  const int t = threadIdx.x;
  const int g = apply_group(nc);
  const int ng = (kk + g - 1) / g;
  // (1) Gram entries u_a^T u_b (a < b) of every group, as dot products over tile rows
  //     from u_b's pivot down (CR rows hold only pivots, which never overlap)
  const int npair = (g * (g - 1)) / 2;
  const int nout = ng * npair;
  if (nout > 0) {
    const int Gr = max(1, NT / nout);
    if (t < Gr * nout) {
      const int o = t % nout, gr = t / nout;
      const int gi = o / npair, pi = o - gi * npair;
      // pair index pi -> (a, b), a < b
      int a = 0, bb = 1, cnt = pi;
      while (cnt >= bb) {
        cnt -= bb;
        ++bb;
      }
      a = cnt;
      const int ja = gi * g + a, jb = gi * g + bb;
      T acc = T(0);
      if (jb < kk) {
        const int start = jb < k ? 0 : jb - k;
        if constexpr (is_df<T>::value) {
          float sh = 0.f, sl = 0.f;
          for (int r = start + gr; r < M; r += Gr)
            df_dot_acc(sh, sl, refl_entry(V, ldv, k, ja, r), refl_entry(V, ldv, k, jb, r));
          acc = df_finish(sh, sl);
        } else {
          for (int r = start + gr; r < M; r += Gr) acc += refl_entry(V, ldv, k, ja, r) * refl_entry(V, ldv, k, jb, r);
        }
      }
      s.red[gr * nout + o] = acc;
    }
    __syncthreads();
    if (t < nout) {
      const int Gr = max(1, NT / nout);
      T sum = s.red[t];
      for (int gr = 1; gr < Gr; ++gr) sum += s.red[gr * nout + t];
      s.red[t] = sum;
    }
    __syncthreads();
  }
  // (2) T of every group (one thread per group), packed upper triangles of 10 entries
  for (int gi = t; gi < ng; gi += NT) {
    T *Tg = Tst + gi * 10;
    const T *Gp = s.red + gi * npair;
    const int gs = min(g, kk - gi * g);
    for (int i = 0; i < gs; ++i) {
      const T ti = tau[gi * g + i];
      Tg[tri_idx(i, i)] = ti;
      for (int a = 0; a < i; ++a) {
        // T(a, i) = -tau_i sum_{a <= c < i} T(a, c) G(c, i)
        T acc = T(0);
        for (int c = a; c < i; ++c) acc += Tg[tri_idx(a, c)] * Gp[tri_idx(c, i) - i];
        Tg[tri_idx(a, i)] = -(ti * acc);
      }
    }
  }
  __syncthreads();
  // (3) groups from the last to the first (Q_t = H_0 ... H_{kk-1} acts on C from the right end)
  for (int gi = ng - 1; gi >= 0; --gi) {
    const int j0 = gi * g, gs = min(g, kk - j0);
    const int nd = gs * nc;
    const int Gr = max(1, NT / nd);
    const T *Tg = Tst + gi * 10;
    // (3a) D = U^T C: output o = (i, c), row groups gr
    if (t < Gr * nd) {
      const int o = t % nd, gr = t / nd;
      const int i = o % gs, c = o / gs;
      const int j = j0 + i;
      const int start = j < k ? 0 : j - k;
      T acc = T(0);
      if constexpr (is_df<T>::value) {
        float sh = 0.f, sl = 0.f;
        for (int r = start + gr; r < M; r += Gr)
          df_dot_acc(sh, sl, refl_entry(V, ldv, k, j, r), CT[(size_t)r * ldct + c]);
        acc = df_finish(sh, sl);
      } else {
        for (int r = start + gr; r < M; r += Gr) acc += refl_entry(V, ldv, k, j, r) * CT[(size_t)r * ldct + c];
      }
      if (gr == 0 && j < k) acc += CR[(size_t)j * ldcr + c];
      s.red[gr * nd + o] = acc;
    }
    __syncthreads();
    // (3b) W = T D: thread (i, c) sums the partials of D(i'..gs-1, c) it needs
    if (t < nd) {
      const int i = t % gs, c = t / gs;
      T w = T(0);
      for (int i2 = i; i2 < gs; ++i2) {
        const int o2 = i2 + gs * c;
        T d = s.red[o2];
        for (int gr = 1; gr < Gr; ++gr) d += s.red[gr * nd + o2];
        w += Tg[tri_idx(i, i2)] * d;
      }
      s.wbuf[t] = w;
    }
    __syncthreads();
    // (3c) C -= U W
    if (t < nd) {
      const int i = t % gs, c = t / gs;
      if (j0 + i < k) CR[(size_t)(j0 + i) * ldcr + c] -= s.wbuf[t];
    }
    {
      const int rstart = j0 < k ? 0 : j0 - k;
      const int q = NT / nc;  // threads per column
      if (t < q * nc) {
        const int c = t % nc;
        const T w0 = s.wbuf[gs * c], w1 = gs > 1 ? s.wbuf[1 + gs * c] : T(0);
        const T w2 = gs > 2 ? s.wbuf[2 + gs * c] : T(0), w3 = gs > 3 ? s.wbuf[3 + gs * c] : T(0);
        auto sub = [](T x, T v, T w) -> T {
          if constexpr (is_df<T>::value)
            return df_sub_prod(x, v, w);
          else
            return x - v * w;
        };
        for (int r = rstart + t / nc; r < M; r += q) {
          T x = CT[(size_t)r * ldct + c];
          x = sub(x, refl_entry(V, ldv, k, j0, r), w0);
          if (gs > 1) x = sub(x, refl_entry(V, ldv, k, j0 + 1, r), w1);
          if (gs > 2) x = sub(x, refl_entry(V, ldv, k, j0 + 2, r), w2);
          if (gs > 3) x = sub(x, refl_entry(V, ldv, k, j0 + 3, r), w3);
          CT[(size_t)r * ldct + c] = x;
        }
      }
    }
    __syncthreads();
  }
}

__device__ __host__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Row range of leaf p when I slices are split over P leaves.
__device__ __host__ __forceinline__ int64_t leaf_begin(int64_t I, int P, int p) { return (int64_t)p * I / P; }

}  // namespace ttgb
