// tt_round.cu -- TT rounding (Alg. 2, organised as the implicit-Q Alg. 6) and the
// orthonormalization norm (Sec. 3.2.4) on one GPU.
//
// Sweep 1 (right-to-left, n = N-1..1, 0-based): for core n the leaf CTAs form the rows
// of A = H(X_n x_3 P)^T (P = triangular factor pushed from core n+1; the push is the
// TRMM of Alg. 6 fused into the slab load) and factor them; a tree of node CTAs reduces
// the leaf triangles to R_n, which becomes P for core n-1.  Reflectors stay stored.
// Sweep 2 (left-to-right, n = 0..N-2): the leaf CTAs of core n apply the stored Q_n to
// [C_p; 0] (C = S_{n-1}^T passed down the tree; TSQR-Apply-Q, Alg. 4) to obtain slabs of
// Y_n = S_{n-1} x_1 Q_n, transpose each slab into rows of V(Y_n) and factor those (second
// TSQR of Alg. 6); the root factor gets an FP64 one-sided Jacobi SVD and the rank rule
// sum_{j>L} sigma_j^2 <= delta^2; the output core is Q' [U_hat; 0] and Sigma V^T moves on.
// The last core is S_{N-2} x_1 Q_{N-1}.
//
// Every size that depends on data (the new ranks) is read by the kernels from a device
// control block, so no step needs a host synchronization; grids depend on shapes only.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tt.h"
#include "tt_internal.cuh"
#include "tt_engine.h"

namespace ttgb {

// ------------------------------------------------------------------------------------
// kernel argument blocks
// ------------------------------------------------------------------------------------

struct Geom {
  int64_t I;  // slices of the core
  int P;      // leaves
  int Tt;     // slices per tile
};

// Source of an input core's entries (a, i, c): a stored core (R0 x I x R1, entry at
// a + R0 (i + I c)), or the Hadamard product of two stored cores A_n, B_n (Sec. 3.2.2)
// formed on the fly, so that the rounding of A o B never writes or reads the
// R_A R_B x I x R_A' R_B' product: row a = p Rb + q and column c = s Rb' + t of slice i
// give A_n(p, i, s) B_n(q, i, t).
template <typename S>
struct CoreSrc {
  const S *X = nullptr;  // the core, or A_n
  const S *B = nullptr;  // B_n (Hadamard), else nullptr
  int R0 = 1;            // left rank of the (product) core
  int ra0 = 1, rb0 = 1, rb1 = 1;
  int64_t I = 1;
};

template <typename T, typename S>
__device__ __forceinline__ T src_load(const CoreSrc<S> &s, int64_t a, int64_t i, int64_t c) {
  if (!s.B) return T(s.X[(size_t)a + (size_t)s.R0 * ((size_t)i + (size_t)s.I * c)]);
  const int64_t p = a / s.rb0, q = a - p * s.rb0, sa = c / s.rb1, tb = c - sa * s.rb1;
  const S va = s.X[(size_t)p + (size_t)s.ra0 * ((size_t)i + (size_t)s.I * sa)];
  const S vb = s.B[(size_t)q + (size_t)s.rb0 * ((size_t)i + (size_t)s.I * tb)];
  if constexpr (std::is_same<T, float>::value)
    return va * vb;
  else
    return T((double)va * (double)vb);  // exact for FP32 factors (held as a double-float pair)
}

template <typename S, typename T>
struct S1Args {
  CoreSrc<S> X;  // core n: b x I x cin
  Geom g;
  int b, cin, rho;   // columns (R_n), right rank of X (R_{n+1}), rows per slice (K_{n+1})
  const double *Pm;  // rho x cin row-major (upper trapezoidal), nullptr = identity (rho == cin == 1)
  T *refl;           // (I*rho) x b row-major
  T *tau;            // I x b
  double *Rleaf;     // P x b*b row-major
  int CC;            // push chunk width
  // shared-memory offsets (bytes); a negative offset -1-e places the buffer at element e
  // of this leaf's region of the global scratch (used when shared memory is short)
  int oRr, oTile, oXs, oPs, oRed, oW, oSc, oTau;
  int ldt;
  T *gscr;
  size_t gstride;
  const float2 *Pm32;  // Pm split into FP32 pairs (hi, lo), for the FP32-storage types
  int stage_p;         // FP32-storage types: 1 = stage Pm32 in shared memory (oPs), 0 = read it via L1
};

struct TreeArgs {
  const double *Rin;  // children R's (b*b each) -- factor
  double *Rout;       // node R's -- factor
  const double *Cin;  // node C's (b*ldc each) -- apply
  double *Cout;       // children C's -- apply
  double *slots;      // per child: MT-row chunks of reflectors (b*b) + taus (nchunk*b)
  int nchild, G, b, MT, nchunk;
  int64_t I;
  int P;
  int lpc;               // leaves per child
  int rho;               // rows per slice (if rho_dyn == nullptr)
  const int *rho_dyn;    // rows per slice read from the control block
  int ncol;              // columns of C (if ncol_dyn == nullptr)
  const int *ncol_dyn;
  int ldc;               // leading dimension of C blocks
  int oA, oB, oRed, oW, oSc, oTau;  // smem offsets
  int lda;
};

template <typename S, typename T>
struct S2Args {
  // mode A (core n >= 1): apply stored sweep-1 Q_n to C; mode B (core 0): push X_0
  int mode;       // 0 = A, 1 = B, 2 = last core (mode A, write output, no V-QR),
                  // 3 = explicit orthonormal factor (mode 2 for any K1, unscaled)
  Geom g;
  // mode A
  const T *qrefl;       // (I*K1) x b1 (sweep-1 reflectors)
  const T *qtau;        // I x b1
  int b1;               // columns of the sweep-1 QR (R_n)
  int K1;               // rows per slice of the sweep-1 QR = columns of the V-QR (K_{n+1})
  const double *Cleaf;  // per leaf: C (k_leaf x L) with leading dim ldc
  int ldc;
  const int *Lcur;      // &L[n]: columns of C = rows per slice of V(Y_n)
  // mode B
  CoreSrc<S> X0;        // core 0: 1 x I x cin
  int cin;
  const double *Pm;     // K1 x cin
  int CC;
  // outputs
  T *vrefl;             // (I*L) x K1 (V-QR reflectors)
  T *vtau;              // I x K1
  double *Rleaf;        // P x K1*K1
  S *out;               // last core output (L x I x 1)
  const int *E;         // exponent gathered by the sweep-1 rescaling (see out_scale)
  int n, N;             // index of the core written, number of cores
  int oQ, oCT, oCR, oRr, oXs, oPs, oRed, oW, oSc, oTq, oTv, oTs;
  int ldq, ldv;
  T *gscr;
  size_t gstride;
};

template <typename S, typename T>
struct OutArgs {
  Geom g;
  const T *vrefl;
  const T *vtau;
  int K1;
  const int *Lcur;      // &L[n]
  const int *Lnext;     // &L[n+1]
  const double *Uleaf;  // per leaf: U (k'_leaf x Lnext), leading dim ldc
  int ldc;
  S *out;               // output core n: L[n] x I x L[n+1]
  const int *E;         // exponent gathered by the sweep-1 rescaling (see out_scale)
  int n, N;
  int oV, oCT, oCR, oRed, oW, oSc, oTau, oTs;
  int ldv;
  T *gscr;
  size_t gstride;
};

struct SvdArgs {
  const double *Rroot;  // K x K row-major
  int K;                // columns
  int64_t In;           // slices of core n
  const int *Lcur;      // &L[n]
  int *Lnext;           // &L[n+1]
  int n, N;
  double eps;
  double *scal;         // [0] = ||X||, [1] = delta in the rescaled units of the sweep
  const int *E;         // exponent gathered by the sweep-1 rescaling: ||X|| = 2^E ||X~_1||
  double *Uhat;         // k_root x K (ld ldu)
  double *Cnext;        // K x K (ld ldu)
  int ldu;
  int *status;
  int precond;          // run the FP32 pre-sweeps (shared memory permitting)
  double *Vg;           // K x K rotation accumulator in global memory when the shared memory
                        // holds only A (ranks above ~117), else nullptr
};

// ------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T *sm(unsigned char *base, int off) {
  return reinterpret_cast<T *>(base + off);
}

__device__ __forceinline__ int dyn(const int *p, int v) { return p ? *p : v; }

// buffer at shared offset off, or (off < 0) at element -1-off of this CTA's global scratch
template <typename T>
__device__ __forceinline__ T *buf(unsigned char *base, int off, T *gscr, size_t gstride) {
  return off >= 0 ? reinterpret_cast<T *>(base + off) : gscr + (size_t)blockIdx.x * gstride + (size_t)(-1 - off);
}

// buf with the spill mode known at compile time: without spilling the compiler sees shared
// memory and issues shared loads (generic loads measured ~20 % slower in the FP32-storage
// sweep-2 kernels)
template <bool SP, typename T>
__device__ __forceinline__ T *sbuf(unsigned char *base, int off, T *gscr, size_t gstride) {
  if constexpr (SP)
    return buf<T>(base, off, gscr, gstride);
  else
    return reinterpret_cast<T *>(base + off);
}

// rows of the stacked matrix owned by leaf range [l0, l1)
__device__ __forceinline__ int64_t rows_of_leaves(int64_t I, int P, int l0, int l1, int rho) {
  return (leaf_begin(I, P, l1) - leaf_begin(I, P, l0)) * (int64_t)rho;
}

// ------------------------------------------------------------------------------------
// sweep 1 leaf: push + sequential Householder over tiles
// ------------------------------------------------------------------------------------

// an entry of the pushed factor in the compute type
__device__ __forceinline__ double load_pm(const double *P, int i, double) { return P[i]; }
__device__ __forceinline__ df32 load_pm(const float2 *P, int i, df32) {
  const float2 v = P[i];
  return df32(v.x, v.y);
}
__device__ __forceinline__ float load_pm(const float2 *P, int i, float) { return P[i].x; }

template <typename S, typename T>
__global__ void __launch_bounds__(NT) k_s1_leaf(S1Args<S, T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *Rr = buf<T>(smem, a.oRr, a.gscr, a.gstride), *tile = sm<T>(smem, a.oTile), *Xs = sm<T>(smem, a.oXs);
  T *Ps = buf<T>(smem, a.oPs, a.gscr, a.gstride);
  Scratch<T> s{sm<T>(smem, a.oRed), sm<T>(smem, a.oW), sm<T>(smem, a.oSc)};
  T *taus = sm<T>(smem, a.oTau);
  const int p = blockIdx.x, t = threadIdx.x;
  const int b = a.b, rho = a.rho, cin = a.cin, ldt = a.ldt;
  const int64_t s0 = leaf_begin(a.g.I, a.g.P, p), s1 = leaf_begin(a.g.I, a.g.P, p + 1);
  const bool push = a.Pm != nullptr;
  // The pushed factor: FP64 reads it through L1 as is.  The FP32-storage types stage its
  // (hi, lo) split in shared memory when two leaf CTAs still fit on an SM with it, and
  // read the split through L1 otherwise (the staged copy would halve the resident CTAs).
  constexpr bool stage = !std::is_same<T, double>::value;
  if (push && stage && a.stage_p)
    for (int idx = t; idx < rho * cin; idx += NT) Ps[idx] = load_pm(a.Pm32, idx, T());
  for (int idx = t; idx < b * b; idx += NT) Rr[idx] = T(0);
  __syncthreads();
  int k = 0;
  for (int64_t i0 = s0; i0 < s1; i0 += a.g.Tt) {
    const int nt = (int)min((int64_t)a.g.Tt, s1 - i0);
    const int M = nt * rho;
    if (!push) {
      // rho == cin == 1: the tile rows are the slices themselves
      for (int idx = t; idx < M * b; idx += NT) {
        const int r = idx / b, c = idx - r * b;
        tile[r * ldt + c] = src_load<T>(a.X, c, i0 + r, 0);
      }
    } else {
      for (int idx = t; idx < M * b; idx += NT) {
        const int r = idx / b, c = idx - r * b;
        tile[r * ldt + c] = T(0);
      }
      for (int c0 = 0; c0 < cin; c0 += a.CC) {
        const int cc_n = min(a.CC, cin - c0);
        __syncthreads();
        const int chunk = nt * b;
        for (int idx = t; idx < cc_n * chunk; idx += NT) {
          const int cc = idx / chunk, rem = idx - cc * chunk;
          if (!a.X.B) {
            Xs[idx] = T(a.X.X[(size_t)b * (i0 + (int64_t)a.g.I * (c0 + cc)) + rem]);
          } else {
            const int il = rem / b;
            Xs[idx] = src_load<T>(a.X, rem - il * b, i0 + il, c0 + cc);
          }
        }
        __syncthreads();
        // one copy of the loop per place the factor is read from (FP64 global, staged
        // shared copy, or the (hi, lo) split in global memory)
        auto push_tile = [&](const T *P) {
          for (int idx = t; idx < M * b; idx += NT) {
            const int r = idx / b, col = idx - r * b;
            const int sl = r / rho, kr = r - sl * rho;
            T acc = tile[r * ldt + col];
            const int cstart = max(kr, c0);
            if constexpr (is_df<T>::value) {
              float ah = acc.hi, al = acc.lo;
              for (int c = cstart; c < c0 + cc_n; ++c) df_dot_acc(ah, al, P[kr * cin + c], Xs[((c - c0) * nt + sl) * b + col]);
              acc = df_finish(ah, al);
            } else {
              for (int c = cstart; c < c0 + cc_n; ++c) acc += P[kr * cin + c] * Xs[((c - c0) * nt + sl) * b + col];
            }
            tile[r * ldt + col] = acc;
          }
        };
        if constexpr (!stage) {
          push_tile(reinterpret_cast<const T *>(a.Pm));
        } else {
          auto push_split = [&](const float2 *P) {
            for (int idx = t; idx < M * b; idx += NT) {
              const int r = idx / b, col = idx - r * b;
              const int sl = r / rho, kr = r - sl * rho;
              T acc = tile[r * ldt + col];
              const int cstart = max(kr, c0);
              if constexpr (is_df<T>::value) {
                float ah = acc.hi, al = acc.lo;
                for (int c = cstart; c < c0 + cc_n; ++c)
                  df_dot_acc(ah, al, load_pm(P, kr * cin + c, T()), Xs[((c - c0) * nt + sl) * b + col]);
                acc = df_finish(ah, al);
              } else {
                for (int c = cstart; c < c0 + cc_n; ++c)
                  acc += load_pm(P, kr * cin + c, T()) * Xs[((c - c0) * nt + sl) * b + col];
              }
              tile[r * ldt + col] = acc;
            }
          };
          if (!a.stage_p)
            push_split(a.Pm32);
          else if (a.oPs >= 0)
            push_tile(sm<T>(smem, a.oPs));
          else
            push_tile(Ps);
        }
      }
    }
    __syncthreads();
    const int kk = hh_factor(Rr, b, k, tile, ldt, M, b, taus, s);
    // store reflectors and taus (the orthonormalization norm needs only R: refl == nullptr)
    if (a.refl) {
      T *dst = a.refl + (size_t)i0 * rho * b;
      for (int idx = t; idx < M * b; idx += NT) {
        const int r = idx / b, c = idx - r * b;
        dst[idx] = tile[r * ldt + c];
      }
      for (int j = t; j < kk; j += NT) a.tau[(size_t)i0 * b + j] = taus[j];
    }
    hh_take_rows(Rr, b, k, kk, tile, ldt, b);
    k = kk;
  }
  double *Ro = a.Rleaf + (size_t)p * b * b;
  for (int idx = t; idx < b * b; idx += NT) Ro[idx] = (idx / b) < k ? (double)Rr[idx] : 0.0;
}

// ------------------------------------------------------------------------------------
// tree: factor one level (children R -> node R), apply one level (node C -> children C)
// ------------------------------------------------------------------------------------

__device__ __forceinline__ int child_rows_k(const TreeArgs &a, int c, int rho) {
  const int l0 = c * a.lpc, l1 = min(a.P, (c + 1) * a.lpc);
  const int64_t rows = rows_of_leaves(a.I, a.P, l0, l1, rho);
  return (int)min64(rows, a.b);
}

// A node whose children all carry full b x b triangles, with more than one triangle to
// stack under the first and room for all of them in one tile, is factored (and applied)
// in one pass over the interleaved triangles; any other node takes its children one by
// one.  Factor and apply decide alike from the same arguments.
__device__ __forceinline__ bool interleaved_node(const TreeArgs &a, int c0, int c1, int rho) {
  if (c1 - c0 < 3 || (c1 - c0 - 1) * a.b > a.MT) return false;
  for (int c = c0; c < c1; ++c)
    if (child_rows_k(a, c, rho) != a.b) return false;
  return true;
}

__global__ void __launch_bounds__(NT) k_tree_factor(TreeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  double *Rr = sm<double>(smem, a.oA), *tile = sm<double>(smem, a.oB);
  Scratch<double> s{sm<double>(smem, a.oRed), sm<double>(smem, a.oW), sm<double>(smem, a.oSc)};
  double *taus = sm<double>(smem, a.oTau);
  const int q = blockIdx.x, t = threadIdx.x, b = a.b;
  const int rho = dyn(a.rho_dyn, a.rho);
  const int c0 = q * a.G, c1 = min(a.nchild, c0 + a.G);
  int k = child_rows_k(a, c0, rho);
  const double *R0 = a.Rin + (size_t)c0 * b * b;
  for (int idx = t; idx < b * b; idx += NT) Rr[idx] = (idx / b) < k ? R0[idx] : 0.0;
  if (interleaved_node(a, c0, c1, rho)) {
    // all children full: the other q = c1 - c0 - 1 triangles, interleaved row by row, form
    // one tile factored in a single pass of b reflectors
    const int qq = c1 - c0 - 1, M = qq * b;
    for (int idx = t; idx < M * b; idx += NT) {
      const int row = idx / b, col = idx - row * b;
      const int r = row / qq, i = row - r * qq;
      tile[row * a.lda + col] = a.Rin[(size_t)(c0 + 1 + i) * b * b + (size_t)r * b + col];
    }
    __syncthreads();
    hh_factor(Rr, b, b, tile, a.lda, M, b, taus, s, 0, qq);
    if (a.slots) {
      for (int idx = t; idx < M * b; idx += NT) {
        const int row = idx / b, col = idx - row * b;
        const int r = row / qq, i = row - r * qq;
        a.slots[(size_t)(c0 + 1 + i) * (b * b + a.nchunk * b) + (size_t)r * b + col] = tile[row * a.lda + col];
      }
      for (int j = t; j < b; j += NT) a.slots[(size_t)(c0 + 1) * (b * b + a.nchunk * b) + (size_t)b * b + j] = taus[j];
    }
    __syncthreads();
    double *Ro = a.Rout + (size_t)q * b * b;
    for (int idx = t; idx < b * b; idx += NT) Ro[idx] = Rr[idx];
    return;
  }
  __syncthreads();
  for (int c = c0 + 1; c < c1; ++c) {
    const int kc = child_rows_k(a, c, rho);
    const double *Rc = a.Rin + (size_t)c * b * b;
    double *slot = a.slots ? a.slots + (size_t)c * (b * b + a.nchunk * b) : nullptr;
    for (int ch = 0, ra = 0; ra < kc; ++ch, ra += a.MT) {
      const int M = min(a.MT, kc - ra);
      for (int idx = t; idx < M * b; idx += NT) {
        const int r = idx / b, col = idx - r * b;
        tile[r * a.lda + col] = Rc[(size_t)(ra + r) * b + col];
      }
      __syncthreads();
      const int kk = hh_factor(Rr, b, k, tile, a.lda, M, b, taus, s, ra);
      if (a.slots) {
        for (int idx = t; idx < M * b; idx += NT) {
          const int r = idx / b, col = idx - r * b;
          slot[(size_t)(ra + r) * b + col] = tile[r * a.lda + col];
        }
        for (int j = t; j < b; j += NT) slot[(size_t)b * b + ch * b + j] = j < kk ? taus[j] : 0.0;
      }
      hh_take_rows(Rr, b, k, kk, tile, a.lda, b);
      k = kk;
    }
  }
  double *Ro = a.Rout + (size_t)q * b * b;
  for (int idx = t; idx < b * b; idx += NT) Ro[idx] = (idx / b) < k ? Rr[idx] : 0.0;
}

__global__ void __launch_bounds__(NT) k_tree_apply(TreeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  double *C = sm<double>(smem, a.oA), *V = sm<double>(smem, a.oB);
  Scratch<double> s{sm<double>(smem, a.oRed), sm<double>(smem, a.oW), sm<double>(smem, a.oSc)};
  double *taus = sm<double>(smem, a.oTau);
  // CT lives right after V (MT x ncol)
  const int q = blockIdx.x, t = threadIdx.x, b = a.b;
  const int rho = dyn(a.rho_dyn, a.rho);
  // the columns of C are independent under Q: CTA y of the node takes columns [cb, cb + nc)
  const int ncol = dyn(a.ncol_dyn, a.ncol);
  const int chunk = (ncol + gridDim.y - 1) / gridDim.y;
  const int cb = blockIdx.y * chunk, nc = min(ncol, cb + chunk) - cb;
  if (nc <= 0) return;
  double *CT = V + (size_t)a.MT * a.lda;
  const int c0 = q * a.G, c1 = min(a.nchild, c0 + a.G);
  // replay the k sequence of the factorization
  int kseq[64 + 1];  // k before each (child, chunk) step; G * nchunk <= 64 enforced by the host
  int nsteps = 0;
  int k = child_rows_k(a, c0, rho);
  for (int c = c0 + 1; c < c1; ++c) {
    const int kc = child_rows_k(a, c, rho);
    for (int ra = 0; ra < kc; ra += a.MT) {
      kseq[nsteps++] = k;
      k = min(k + min(a.MT, kc - ra), b);
    }
  }
  // load node C (k rows)
  const double *Cn = a.Cin + (size_t)q * b * a.ldc + cb;
  for (int idx = t; idx < b * nc; idx += NT) {
    const int r = idx / nc, col = idx - r * nc;
    C[r * nc + col] = r < k ? Cn[(size_t)r * a.ldc + col] : 0.0;
  }
  if (interleaved_node(a, c0, c1, rho)) {
    // Q [C; 0] with the interleaved tile of the factorization; child c0 + 1 + i receives
    // rows r q + i of the lower block, child c0 the upper block
    const int qq = c1 - c0 - 1, M = qq * b;
    for (int idx = t; idx < M * b; idx += NT) {
      const int row = idx / b, col = idx - row * b;
      const int r = row / qq, i = row - r * qq;
      V[row * a.lda + col] = a.slots[(size_t)(c0 + 1 + i) * (b * b + a.nchunk * b) + (size_t)r * b + col];
    }
    for (int j = t; j < b; j += NT) taus[j] = a.slots[(size_t)(c0 + 1) * (b * b + a.nchunk * b) + (size_t)b * b + j];
    for (int idx = t; idx < M * nc; idx += NT) CT[idx] = 0.0;
    __syncthreads();
    hh_apply(V, a.lda, taus, b, M, b, C, nc, CT, nc, nc, s, 0, qq);
    __syncthreads();
    for (int idx = t; idx < M * nc; idx += NT) {
      const int row = idx / nc, col = idx - row * nc;
      const int r = row / qq, i = row - r * qq;
      a.Cout[(size_t)(c0 + 1 + i) * b * a.ldc + (size_t)r * a.ldc + cb + col] = CT[idx];
    }
    double *Cc0 = a.Cout + (size_t)c0 * b * a.ldc + cb;
    for (int idx = t; idx < b * nc; idx += NT) {
      const int r = idx / nc, col = idx - r * nc;
      Cc0[(size_t)r * a.ldc + col] = C[r * nc + col];
    }
    return;
  }
  __syncthreads();
  int step = nsteps;
  for (int c = c1 - 1; c > c0; --c) {
    const int kc = child_rows_k(a, c, rho);
    const double *slot = a.slots + (size_t)c * (b * b + a.nchunk * b);
    double *Cc = a.Cout + (size_t)c * b * a.ldc + cb;
    const int nch = (kc + a.MT - 1) / a.MT;
    for (int ch = nch - 1; ch >= 0; --ch) {
      const int ra = ch * a.MT, M = min(a.MT, kc - ra);
      const int kb = kseq[--step], ka = min(kb + M, b);
      for (int idx = t; idx < M * b; idx += NT) {
        const int r = idx / b, col = idx - r * b;
        V[r * a.lda + col] = slot[(size_t)(ra + r) * b + col];
      }
      for (int j = t; j < b; j += NT) taus[j] = slot[(size_t)b * b + ch * b + j];
      for (int idx = t; idx < M * nc; idx += NT) {
        const int r = idx / nc, col = idx - r * nc;
        CT[r * nc + col] = (kb + r < ka) ? C[(kb + r) * nc + col] : 0.0;
      }
      __syncthreads();
      hh_apply(V, a.lda, taus, kb, M, b, C, nc, CT, nc, nc, s, ra);
      __syncthreads();
      for (int idx = t; idx < M * nc; idx += NT) {
        const int r = idx / nc, col = idx - r * nc;
        Cc[(size_t)(ra + r) * a.ldc + col] = CT[r * nc + col];
      }
      __syncthreads();
    }
  }
  // first child keeps the remaining rows
  const int k0 = child_rows_k(a, c0, rho);
  double *Cc = a.Cout + (size_t)c0 * b * a.ldc + cb;
  for (int idx = t; idx < k0 * nc; idx += NT) {
    const int r = idx / nc, col = idx - r * nc;
    Cc[(size_t)r * a.ldc + col] = C[r * nc + col];
  }
}

// ------------------------------------------------------------------------------------
// sweep 2 leaf: (A) apply Q_n to C_p, form Y_n slabs, factor V(Y_n) slabs
//               (B) core 0: push and factor V(X_0 x_3 P)
//               (last) apply Q_{N-1} and write the last output core
// ------------------------------------------------------------------------------------

// Factor 2^sh that output core n (of N) takes from the exponent E gathered by the sweep-1
// rescaling.  The last core takes all of it when the storage type holds 2^E comfortably
// (always in FP64); in FP32 storage a larger |E| is spread over the cores in near-equal
// integer parts summing to E, so that no stored core leaves the FP32 range (the cores
// before the last are then orthonormal up to their power-of-two factor).
template <typename S>
__device__ __forceinline__ S out_scale(const int *E, int n, int N) {
  const int e = E ? *E : 0;
  int sh;
  if (sizeof(S) == 8 || (e >= -64 && e <= 64))
    sh = n == N - 1 ? e : 0;
  else
    sh = (int)(((int64_t)e * (n + 1)) / N - ((int64_t)e * n) / N);
  return (S)ldexp(1.0, sh);
}

template <typename S, typename T, bool SP>
__global__ void __launch_bounds__(NT) k_s2_leaf(S2Args<S, T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *Q = sm<T>(smem, a.oQ), *CT = sbuf<SP>(smem, a.oCT, a.gscr, a.gstride);
  T *CR = sbuf<SP>(smem, a.oCR, a.gscr, a.gstride), *Rr = sbuf<SP>(smem, a.oRr, a.gscr, a.gstride);
  T *Xs = sm<T>(smem, a.oXs), *Ps = sbuf<SP>(smem, a.oPs, a.gscr, a.gstride);
  Scratch<T> s{sm<T>(smem, a.oRed), sbuf<SP>(smem, a.oW, a.gscr, a.gstride), sm<T>(smem, a.oSc)};
  T *tq = sm<T>(smem, a.oTq), *tv = sm<T>(smem, a.oTv);
  const int p = blockIdx.x, t = threadIdx.x;
  const int64_t s0 = leaf_begin(a.g.I, a.g.P, p), s1 = leaf_begin(a.g.I, a.g.P, p + 1);
  const int K1 = a.K1;
  const int L = a.mode == 1 ? 1 : *a.Lcur;  // rows per slice of V(Y_n)
  const int b1 = a.b1;
  const S osc = a.mode == 2 ? out_scale<S>(a.E, a.n, a.N) : S(1);
  // number of sweep-1 reflector rows owned by this leaf, and its C rows
  int kq = 0;
  if (a.mode != 1) {
    kq = (int)min64((s1 - s0) * (int64_t)K1, b1);
    const double *Cp = a.Cleaf + (size_t)p * b1 * a.ldc;
    for (int idx = t; idx < b1 * L; idx += NT) {
      const int r = idx / L, c = idx - r * L;
      CR[idx] = r < kq ? (T)Cp[(size_t)r * a.ldc + c] : T(0);
    }
  } else {
    for (int idx = t; idx < K1 * a.cin; idx += NT) Ps[idx] = (T)a.Pm[idx];
  }
  for (int idx = t; idx < K1 * K1; idx += NT) Rr[idx] = T(0);
  __syncthreads();
  int kv = 0;  // rows of the running V-QR factor
  // tiles in reverse slice order
  const int64_t ntiles = (s1 - s0 + a.g.Tt - 1) / a.g.Tt;
  for (int64_t ti = ntiles - 1; ti >= 0; --ti) {
    const int64_t i0 = s0 + ti * a.g.Tt;
    const int nt = (int)min((int64_t)a.g.Tt, s1 - i0);
    int Mv = nt * L;  // rows of this V tile
    if (a.mode != 1) {
      // (1) apply this tile's sweep-1 reflectors to [CR; CT]
      const int M1 = nt * K1;
      const int kb = (int)min64((i0 - s0) * (int64_t)K1, b1);
      const int ka = min(kb + M1, b1);
      const T *src = a.qrefl + (size_t)i0 * K1 * b1;
      for (int idx = t; idx < M1 * b1; idx += NT) {
        const int r = idx / b1, c = idx - r * b1;
        Q[r * a.ldq + c] = src[idx];
      }
      for (int j = t; j < ka; j += NT) tq[j] = a.qtau[(size_t)i0 * b1 + j];
      for (int idx = t; idx < M1 * L; idx += NT) {
        const int r = idx / L, c = idx - r * L;
        CT[idx] = (kb + r < ka) ? CR[(kb + r) * L + c] : T(0);
      }
      __syncthreads();
      hh_apply_grouped(Q, a.ldq, tq, kb, M1, b1, CR, L, CT, L, L, s, sbuf<SP>(smem, a.oTs, a.gscr, a.gstride));
      __syncthreads();
      if (a.mode >= 2) {
        // last core (K1 == 1) or an explicit orthonormal factor: tile row (i - i0) K1 + k
        // of Q_n [C_p; 0] is row (i, k) of H(Y_n)^T, so Y[l, i, k] = CT[(i - i0) K1 + k][l]
        for (int idx = t; idx < nt * K1 * L; idx += NT) {
          const int r = idx / L, l = idx - r * L;
          const int il = r / K1, k = r - il * K1;
          a.out[(size_t)l + (size_t)L * ((i0 + il) + a.g.I * (int64_t)k)] = (S)CT[r * L + l] * osc;
        }
        __syncthreads();
        continue;
      }
      // (2) V tile: row (i - i0) * L + l, column k  <-  CT[(i - i0) * K1 + k][l]   (reuse Q)
      for (int idx = t; idx < Mv * K1; idx += NT) {
        const int r = idx / K1, kc = idx - r * K1;
        const int il = r / L, l = r - il * L;
        Q[r * a.ldv + kc] = CT[(il * K1 + kc) * L + l];
      }
      __syncthreads();
    } else {
      // core 0: V tile row (i - i0), column k = sum_c X0[i + I c] P[k][c]
      for (int idx = t; idx < Mv * K1; idx += NT) Q[(idx / K1) * a.ldv + (idx % K1)] = T(0);
      for (int c0 = 0; c0 < a.cin; c0 += a.CC) {
        const int cc_n = min(a.CC, a.cin - c0);
        __syncthreads();
        for (int idx = t; idx < cc_n * nt; idx += NT) {
          const int cc = idx / nt, il = idx - cc * nt;
          Xs[idx] = src_load<T>(a.X0, 0, i0 + il, c0 + cc);
        }
        __syncthreads();
        for (int idx = t; idx < Mv * K1; idx += NT) {
          const int il = idx / K1, kc = idx - il * K1;
          T acc = Q[il * a.ldv + kc];
          for (int c = max(kc, c0); c < c0 + cc_n; ++c) acc += Ps[kc * a.cin + c] * Xs[(c - c0) * nt + il];
          Q[il * a.ldv + kc] = acc;
        }
      }
      __syncthreads();
    }
    // (3) factor the V tile under the running factor
    const int kk = hh_factor(Rr, K1, kv, Q, a.ldv, Mv, K1, tv, s);
    T *dst = a.vrefl + (size_t)i0 * L * K1;
    for (int idx = t; idx < Mv * K1; idx += NT) {
      const int r = idx / K1, c = idx - r * K1;
      dst[idx] = Q[r * a.ldv + c];
    }
    for (int j = t; j < kk; j += NT) a.vtau[(size_t)i0 * K1 + j] = tv[j];
    hh_take_rows(Rr, K1, kv, kk, Q, a.ldv, K1);
    kv = kk;
  }
  if (a.mode >= 2) return;
  double *Ro = a.Rleaf + (size_t)p * K1 * K1;
  for (int idx = t; idx < K1 * K1; idx += NT) Ro[idx] = (idx / K1) < kv ? (double)Rr[idx] : 0.0;
}

// ------------------------------------------------------------------------------------
// sweep 2 output: core n = Q'_n [U_p; 0]
// ------------------------------------------------------------------------------------

template <typename S, typename T, bool SP>
__global__ void __launch_bounds__(NT) k_s2_out(OutArgs<S, T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *V = sm<T>(smem, a.oV), *CT = sbuf<SP>(smem, a.oCT, a.gscr, a.gstride), *CR = sbuf<SP>(smem, a.oCR, a.gscr, a.gstride);
  Scratch<T> s{sm<T>(smem, a.oRed), sbuf<SP>(smem, a.oW, a.gscr, a.gstride), sm<T>(smem, a.oSc)};
  T *tv = sm<T>(smem, a.oTau);
  const int p = blockIdx.x, t = threadIdx.x;
  const int64_t s0 = leaf_begin(a.g.I, a.g.P, p), s1 = leaf_begin(a.g.I, a.g.P, p + 1);
  const int K1 = a.K1, L = *a.Lcur, Ln = *a.Lnext;
  const S osc = out_scale<S>(a.E, a.n, a.N);
  const int kleaf = (int)min64((s1 - s0) * (int64_t)L, K1);
  const double *Up = a.Uleaf + (size_t)p * K1 * a.ldc;
  for (int idx = t; idx < K1 * Ln; idx += NT) {
    const int r = idx / Ln, c = idx - r * Ln;
    CR[idx] = r < kleaf ? (T)Up[(size_t)r * a.ldc + c] : T(0);
  }
  __syncthreads();
  // the V-QR processed tiles in reverse slice order, so Q' is applied in forward order
  for (int64_t i0 = s0; i0 < s1; i0 += a.g.Tt) {
    const int nt = (int)min((int64_t)a.g.Tt, s1 - i0);
    const int Mv = nt * L;
    const int ka = (int)min64((s1 - i0) * (int64_t)L, K1);
    const int kb = (int)min64((s1 - i0 - nt) * (int64_t)L, K1);
    const T *src = a.vrefl + (size_t)i0 * L * K1;
    for (int idx = t; idx < Mv * K1; idx += NT) {
      const int r = idx / K1, c = idx - r * K1;
      V[r * a.ldv + c] = src[idx];
    }
    for (int j = t; j < ka; j += NT) tv[j] = a.vtau[(size_t)i0 * K1 + j];
    for (int idx = t; idx < Mv * Ln; idx += NT) {
      const int r = idx / Ln, c = idx - r * Ln;
      CT[idx] = (kb + r < ka) ? CR[(kb + r) * Ln + c] : T(0);
    }
    __syncthreads();
    hh_apply_grouped(V, a.ldv, tv, kb, Mv, K1, CR, Ln, CT, Ln, Ln, s, sbuf<SP>(smem, a.oTs, a.gscr, a.gstride));
    __syncthreads();
    // rows (i - i0) * L + l, column l'  ->  out[l + L (i + I l')]
    for (int idx = t; idx < Mv * Ln; idx += NT) {
      const int c = idx / Mv, r = idx - c * Mv;
      a.out[(size_t)L * i0 + r + (size_t)L * a.g.I * c] = (S)CT[r * Ln + c] * osc;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// SVD of the root factor + rank choice (one CTA)
//
// One-sided Jacobi (Hestenes) with a round-robin pair ordering, one warp per pair.
// When shared memory allows, an FP32 pass first rotates a scaled FP32 copy until its
// columns are orthogonal to FP32 accuracy; its rotation matrix is re-orthonormalized in
// FP64 (Newton-Schulz, V <- V (3I - V^T V) / 2, twice) and applied, B = A V, so the FP64
// sweeps that follow start from nearly orthogonal columns and need few sweeps.  The FP64
// sweeps use the same convergence test as a plain one-sided Jacobi
// (|b_p^T b_q| <= tol ||b_p|| ||b_q||), so the singular values keep FP64 accuracy.
// ------------------------------------------------------------------------------------

constexpr int SVD_NT = 512;

// rotation [c s; -s c] zeroing the (p, q) entry of the 2x2 Gram [[al, ga], [ga, be]]:
// with h = be - al, g = 2 ga, r = sqrt(h^2 + g^2): c = sqrt((|h| + r) / (2r)),
// s = sign(h) g / sqrt(2r (|h| + r)) -- the smaller-angle solution t = s / c of
// t^2 + 2 (h / g) t - 1 = 0; h = 0 takes t = 1.
__device__ __forceinline__ void jrot(double al, double be, double ga, double &c, double &sn) {
  const double h = be - al, g = 2.0 * ga;
  if (h == 0.0) {
    c = sn = 0.70710678118654752;
    return;
  }
  const double ah = fabs(h);
  const double x = fma(h, h, g * g);
  const double r = nr_range(x) ? x * rsqrt_nr(x) : sqrt(x);
  const double q = 2.0 * r * (ah + r);
  const double w = nr_range(q) ? rsqrt_nr(q) : 1.0 / sqrt(q);
  c = (ah + r) * w;
  sn = (h > 0.0 ? g : -g) * w;
}

__device__ __forceinline__ void jrot(float al, float be, float ga, float &c, float &sn) {
  const float h = be - al, g = 2.0f * ga;
  if (h == 0.0f) {
    c = sn = 0.70710678f;
    return;
  }
  const float ah = fabsf(h);
  const float r = sqrtf(fmaf(h, h, g * g));
  const float w = rsqrtf(2.0f * r * (ah + r));
  if (!(w < 3.0e38f)) {  // underflowed operands: leave the pair alone
    c = 1.0f;
    sn = 0.0f;
    return;
  }
  c = (ah + r) * w;
  sn = (h > 0.0f ? g : -g) * w;
}


// sum over the LP consecutive lanes of a segment (LP a power of two <= 32)
template <int LP, typename T>
__device__ __forceinline__ T seg_sum(T v) {
#pragma unroll
  for (int o = LP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Round-robin one-sided Jacobi on A (ms x ns, column-major), accumulating the rotations
// into V (ns x ns, column-major).  pos holds 2 * (ns + 2) ints, flag 1 int.  Returns
// whether a sweep completed without rotating.  Pairs whose two columns both have squared
// norms <= neg2 are left alone (deflation of negligible columns), and so are pairs with one
// column of squared norm <= neg1: its coupling g <= |c1| |c2| to the other column moves the
// pair's eigenvalues by at most g^2 / gap <= neg1 and the other column's direction by at
// most sqrt(neg1) in norm, so such a column (rounding noise of a rank-deficient factor)
// cannot keep the sweeps going.
// Each pair is handled by a segment of LP = 8 lanes (4 pairs per warp): on GB300 an FP64
// warp instruction costs the FP64 unit the same time whatever its active lanes, so the
// per-pair dot products, reductions and rotation angle are packed four to an instruction.
// quad_stop: also stop after a sweep whose largest rotated cos^2 = ga^2 / (al be) is at
// most 0.1 tol: cyclic Jacobi converges quadratically (the next sweep's cos^2 is about the
// square of this one's), so the sweep that would only confirm convergence is skipped.
// pos holds 2 * (ns + 2) ints, flag 2 ints.
template <typename T>
__device__ bool jacobi(T *A, T *V, int ms, int ns, int *pos, int *flag, T tol, int maxsweeps, T neg2, T neg1,
                       bool quad_stop = false, bool accumulate_v = true) {
  constexpr int LP = 8, PW = 32 / LP;  // lanes per pair, pairs per warp
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = SVD_NT / 32;
  const int seg = lane / LP, sl = lane - seg * LP;
  if (ns <= 1) return true;
  const int n2 = (ns + 1) & ~1;
  const int stride = ns + 2;
  for (int i = t; i < n2; i += SVD_NT) pos[i] = i;
  __syncthreads();
  int cur = 0;
  const T tol2 = tol * tol;
  for (int sweep = 0; sweep < maxsweeps; ++sweep) {
    if (t == 0) {
      flag[0] = 0;
      flag[1] = 0;  // bits of the largest rotated cos^2 (a non-negative float orders as an int)
    }
    __syncthreads();
    for (int round = 0; round < n2 - 1; ++round) {
      const int *P = pos + cur * stride;
      // every lane of a warp runs the same number of iterations (the shuffles need the
      // whole warp); segments without a pair in an iteration compute on dummy values
      for (int base = warp * PW; base < n2 / 2; base += nwarp * PW) {
        const int pr = base + seg;
        int pp = pr < n2 / 2 ? P[pr] : ns, qq = pr < n2 / 2 ? P[n2 - 1 - pr] : ns;
        const bool live = pp < ns && qq < ns;
        if (pp > qq) {
          const int tmp = pp;
          pp = qq;
          qq = tmp;
        }
        T *bp = A + (size_t)(live ? pp : 0) * ms, *bq = A + (size_t)(live ? qq : 0) * ms;
        T al = 0, be = 0, ga = 0;
        if (live) {
          for (int r = sl; r < ms; r += LP) {
            const T x = bp[r], y = bq[r];
            al += x * x;
            be += y * y;
            ga += x * y;
          }
        }
        al = seg_sum<LP>(al);
        be = seg_sum<LP>(be);
        ga = seg_sum<LP>(ga);
        if (!live || ga == T(0) || ga * ga <= tol2 * al * be || (al <= neg2 && be <= neg2) || al <= neg1 ||
            be <= neg1)
          continue;
        if (quad_stop && sl == 0) atomicMax(flag + 1, __float_as_int((float)((ga / al) * (ga / be))));
        T cs, sn;
        jrot(al, be, ga, cs, sn);
        for (int r = sl; r < ms; r += LP) {
          const T x = bp[r], y = bq[r];
          bp[r] = cs * x - sn * y;
          bq[r] = sn * x + cs * y;
        }
        if (accumulate_v) {
          T *vp = V + (size_t)pp * ns, *vq = V + (size_t)qq * ns;
          for (int r = sl; r < ns; r += LP) {
            const T x = vp[r], y = vq[r];
            vp[r] = cs * x - sn * y;
            vq[r] = sn * x + cs * y;
          }
        }
        if (sl == 0) flag[0] = 1;
      }
      __syncthreads();
      int *Pn = pos + (cur ^ 1) * stride;
      for (int i = t; i < n2; i += SVD_NT) Pn[i] = i == 0 ? P[0] : (i == 1 ? P[n2 - 1] : P[i - 1]);
      cur ^= 1;
      __syncthreads();
    }
    const int any = flag[0];
    const float cmax = __int_as_float(flag[1]);
    __syncthreads();
    if (!any) return true;
    if (quad_stop && (double)cmax <= 0.1 * (double)tol) return true;
  }
  return false;
}

// shared-memory doubles of the SVD kernel: A, V, work area W, sigma
__host__ __device__ inline size_t svd_w_doubles(int ms, int ns) {
  const size_t a = (size_t)ms * ns, b = 2 * (size_t)ns * ns;
  return a > b ? a : b;
}

// Re-orthonormalizes the nearly orthogonal V (ns x ns, column-major) by Newton-Schulz
// iterations in FP64 (X = V^T V, V <- 1.5 V - 0.5 V X; each squares the departure from
// orthogonality) and replaces A (ms x ns) by A V.  W: 2 ns^2 >= ms ns doubles of scratch.
__device__ void orth_apply(double *A, double *Vm, double *W, int ms, int ns, int iters) {
  const int t = threadIdx.x;
  double *X = W, *Y = W + (size_t)ns * ns;
  for (int it = 0; it < iters; ++it) {
    for (int idx = t; idx < ns * ns; idx += SVD_NT) {
      const int j = idx / ns, i = idx - j * ns;
      double acc = 0.0;
      for (int r = 0; r < ns; ++r) acc += Vm[(size_t)i * ns + r] * Vm[(size_t)j * ns + r];
      X[idx] = acc;
    }
    __syncthreads();
    for (int idx = t; idx < ns * ns; idx += SVD_NT) {
      const int j = idx / ns, r = idx - j * ns;
      double acc = 0.0;
      for (int i = 0; i < ns; ++i) acc += Vm[(size_t)i * ns + r] * X[(size_t)j * ns + i];
      Y[idx] = 1.5 * Vm[idx] - 0.5 * acc;
    }
    __syncthreads();
    for (int idx = t; idx < ns * ns; idx += SVD_NT) Vm[idx] = Y[idx];
    __syncthreads();
  }
  // A V (into W, then back into A)
  for (int idx = t; idx < ms * ns; idx += SVD_NT) {
    const int j = idx / ms, r = idx - j * ms;
    double acc = 0.0;
    for (int i = 0; i < ns; ++i) acc += A[(size_t)i * ms + r] * Vm[(size_t)j * ns + i];
    W[idx] = acc;
  }
  __syncthreads();
  for (int idx = t; idx < ms * ns; idx += SVD_NT) A[idx] = W[idx];
  __syncthreads();
}

__global__ void __launch_bounds__(SVD_NT) k_svd(SvdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = a.K, t = threadIdx.x;
  const int Lc = *a.Lcur;
  const int kroot = (int)min64((int64_t)Lc * a.In, K);
  const bool wide = kroot < K;
  const int ms = K, ns = wide ? kroot : K;  // A is ms x ns, column-major, ms >= ns
  double *A = reinterpret_cast<double *>(smem);
  double *Vm = a.Vg ? a.Vg : A + (size_t)ms * ns;
  double *W = a.Vg ? A + (size_t)ms * ns : Vm + (size_t)ns * ns;
  const bool pre = a.precond != 0;
  double *sig = pre ? W + svd_w_doubles(ms, ns) : W;
  int *pos = reinterpret_cast<int *>(sig + ns);  // 2 * (ns + 2)
  int *ord = pos + 2 * (ns + 2);
  int *flag = ord + ns + 1;                      // 4
  double *red = reinterpret_cast<double *>(flag + 4);  // SVD_NT / 32, 8-aligned below
  red = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(red) + 7) & ~uintptr_t(7));
  for (int idx = t; idx < ms * ns; idx += SVD_NT) {
    const int c = idx / ms, r = idx - c * ms;
    A[idx] = wide ? a.Rroot[(size_t)c * K + r] : a.Rroot[(size_t)r * K + c];
  }
  for (int idx = t; idx < ns * ns; idx += SVD_NT) Vm[idx] = (idx / ns) == (idx % ns) ? 1.0 : 0.0;
  __syncthreads();
  if (pre && ns > 1) {
    // scale by a power of two so the FP32 copy neither over- nor underflows
    double amax = 0.0;
    for (int idx = t; idx < ms * ns; idx += SVD_NT) amax = fmax(amax, fabs(A[idx]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((t & 31) == 0) red[t >> 5] = amax;
    __syncthreads();
    if (t == 0) {
      double m = 0.0;
      for (int w = 0; w < SVD_NT / 32; ++w) m = fmax(m, red[w]);
      red[0] = m;
    }
    __syncthreads();
    amax = red[0];
    __syncthreads();
    if (amax > 0.0 && amax < 1e300) {
      const int ex = (int)((__double_as_longlong(amax) >> 52) & 0x7ff) - 1023;
      const double scl = __longlong_as_double((long long)(1023 - ex) << 52);  // 2^-ex
      float *A32 = reinterpret_cast<float *>(W);
      float *V32 = A32 + (size_t)ms * ns;
      for (int idx = t; idx < ms * ns; idx += SVD_NT) A32[idx] = (float)(A[idx] * scl);
      for (int idx = t; idx < ns * ns; idx += SVD_NT) V32[idx] = (idx / ns) == (idx % ns) ? 1.0f : 0.0f;
      __syncthreads();
      // columns below FP32 resolution relative to the largest entry carry no information here
      jacobi<float>(A32, V32, ms, ns, pos, flag, 4e-6f, 20, 1e-12f * (float)ms, 0.0f);
      int *bad = flag + 2;
      if (t == 0) *bad = 0;
      __syncthreads();
      for (int idx = t; idx < ns * ns; idx += SVD_NT) {
        const double v = (double)V32[idx];
        if (!isfinite(v)) *bad = 1;
        Vm[idx] = v;
      }
      __syncthreads();
      if (*bad) {  // no usable preconditioner: start the FP64 sweeps from V = I
        for (int idx = t; idx < ns * ns; idx += SVD_NT) Vm[idx] = (idx / ns) == (idx % ns) ? 1.0 : 0.0;
      }
      __syncthreads();
      orth_apply(A, Vm, W, ms, ns, 2);
    }
  }
  // Deflation threshold: columns whose squared norm is <= 1e-6 delta^2 / ns can never be
  // kept by the rank rule and their total mass stays exact in the tails (sum of squared
  // column norms), so pairs of two such columns need no rotation; a column of squared norm
  // <= 1e-9 delta^2 / ns needs none with any column (it moves a kept direction by at most
  // 3.2e-5 delta / sqrt(ns), an error below 3.2e-5 eps ||X|| / sqrt(N - 1) in the result).
  // For n = 0, delta is taken from ||A||_F (= ||X||, Sec. 2.3) only to set this threshold.
  {
    double f2 = 0.0;
    if (a.n == 0)
      for (int idx = t; idx < ms * ns; idx += SVD_NT) f2 += A[idx] * A[idx];
    f2 = warp_sum(f2);
    if ((t & 31) == 0) red[t >> 5] = f2;
    __syncthreads();
    if (t == 0) {
      double d2;
      if (a.n == 0) {
        double tot = 0.0;
        for (int w = 0; w < SVD_NT / 32; ++w) tot += red[w];
        d2 = a.N > 1 ? a.eps * a.eps * tot / (double)(a.N - 1) : 0.0;
      } else {
        d2 = a.scal[1] * a.scal[1];
      }
      sig[0] = 1e-6 * d2 / (double)ns;
    }
    __syncthreads();
  }
  const double neg2 = sig[0];
  __syncthreads();
  // A square root factor (not wide) needs no rotation accumulator: the next core's factor
  // V Sigma equals R^T U (R = U Sigma V^T) and is formed from R and U_hat below.
  const bool converged =
      jacobi<double>(A, Vm, ms, ns, pos, flag, 1e-15 * (double)ms, 60, neg2, 1e-3 * neg2, true, wide);
  // singular values
  const int lane = t & 31, warp = t >> 5, nwarp = SVD_NT / 32;
  for (int c = warp; c < ns; c += nwarp) {
    double ss = 0;
    for (int r = lane; r < ms; r += 32) ss += A[(size_t)c * ms + r] * A[(size_t)c * ms + r];
    ss = warp_sum(ss);
    if (lane == 0) sig[c] = sqrt(ss);
  }
  __syncthreads();
  if (t == 0) {
    // stable insertion sort by decreasing sigma
    for (int i = 0; i < ns; ++i) ord[i] = i;
    for (int i = 1; i < ns; ++i) {
      const int key = ord[i];
      int j = i - 1;
      while (j >= 0 && sig[ord[j]] < sig[key]) {
        ord[j + 1] = ord[j];
        --j;
      }
      ord[j + 1] = key;
    }
    bool finite = true;
    for (int i = 0; i < ns; ++i) finite = finite && isfinite(sig[i]);
    if (a.n == 0) {
      double s2 = 0.0;
      for (int i = ns - 1; i >= 0; --i) s2 += sig[ord[i]] * sig[ord[i]];
      const double nrm = sqrt(s2);
      a.scal[0] = ldexp(nrm, *a.E);
      a.scal[1] = a.N > 1 ? a.eps * nrm / sqrt((double)(a.N - 1)) : 0.0;
    }
    const double d2 = a.scal[1] * a.scal[1];
    // L = min{ L >= 1 : tail(L) <= delta^2 }, tail(l) = sum_{j >= l} sigma_j^2 accumulated
    // from the smallest value upward; tail(ns) = 0 always qualifies
    int L = ns;
    double tl = 0.0;
    for (int l = ns - 1; l >= 1; --l) {
      tl += sig[ord[l]] * sig[ord[l]];
      if (tl <= d2)
        L = l;
      else
        break;
    }
    *a.Lnext = L;
    if (!finite || !converged) *a.status = TT_ERR_NUMERICAL;
    flag[1] = L;
  }
  __syncthreads();
  const int L = flag[1];
  for (int idx = t; idx < K * L; idx += SVD_NT) {
    const int r = idx / L, l = idx - r * L;
    const int c = ord[l];
    const double sg = sig[c];
    if (!wide) {
      // R' = U S V^T : U_hat = A(:, c) / sigma (C_next = R'^T U_hat below)
      a.Uhat[(size_t)r * a.ldu + l] = sg > 0.0 ? A[(size_t)c * ms + r] / sg : (r == l ? 1.0 : 0.0);
    } else {
      // R'^T = U' S V'^T : U_hat = V'(:, c) (kroot rows), C_next = A(:, c) (= U' sigma)
      if (r < kroot) a.Uhat[(size_t)r * a.ldu + l] = Vm[(size_t)c * ns + r];
      a.Cnext[(size_t)r * a.ldu + l] = A[(size_t)c * ms + r];
    }
  }
  if (!wide) {
    // C_next(:, l) = V(:, c) sigma_c = R'^T U_hat(:, l) (zero for sigma_c = 0, whose U_hat
    // column is a unit vector, not a singular vector)
    __syncthreads();
    for (int idx = t; idx < K * L; idx += SVD_NT) {
      const int r = idx / L, l = idx - r * L;
      double acc = 0.0;
      if (sig[ord[l]] > 0.0)
        for (int i = 0; i < K; ++i) acc += a.Rroot[(size_t)i * K + r] * a.Uhat[(size_t)i * a.ldu + l];
      a.Cnext[(size_t)r * a.ldu + l] = acc;
    }
  }
}

// ------------------------------------------------------------------------------------
// norm of the pushed first core: sum_{i,k} (sum_c X0[i + I c] P[k][c])^2
// ------------------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(NT) k_push_sumsq(const T *X0, int64_t I, int cin, int K, const double *Pm,
                                                   double *partial) {
  __shared__ double red[NT / 32];
  double acc = 0.0;
  const int64_t total = I * K;
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < total; e += (int64_t)gridDim.x * NT) {
    const int64_t i = e / K;
    const int kk = (int)(e - i * K);
    double v = 0.0;
    if (Pm) {
      for (int c = kk; c < cin; ++c) v += (double)X0[i + I * c] * Pm[kk * cin + c];
    } else {
      v = (double)X0[i];
    }
    acc += v * v;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

// First core of an orthonormalized tensor: Y_0 = 2^E X_0 x_3 P (P = K x cin upper trapezoidal,
// row-major with leading dimension cin: the root factor pushed from core 1, Alg. 1).
template <typename S>
__global__ void __launch_bounds__(NT) k_push_out(const S *X0, int64_t I, int cin, int K, const double *Pm,
                                                 const int *E, S *out) {
  const int64_t total = I * K;
  const double sc = ldexp(1.0, *E);
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < total; e += (int64_t)gridDim.x * NT) {
    const int kk = (int)(e / I);
    const int64_t i = e - (int64_t)kk * I;
    double v = 0.0;
    for (int c = kk; c < cin; ++c) v += (double)X0[i + I * c] * Pm[kk * cin + c];
    out[e] = (S)(v * sc);
  }
}

// C <- identity (k x k, row-major with leading dimension ld)
__global__ void k_eye(double *C, int k, int ld) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < k * k; idx += gridDim.x * blockDim.x) {
    const int r = idx / k, c = idx - r * k;
    C[(size_t)r * ld + c] = r == c ? 1.0 : 0.0;
  }
}

__global__ void k_set_int(int *p, int v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

__global__ void k_init_ctl(int *L, int N, int *status) {
  for (int i = threadIdx.x; i <= N; i += blockDim.x) L[i] = 1;
  if (threadIdx.x < 4) status[threadIdx.x] = 0;
}

__global__ void k_sum_sqrt(const double *partial, int n, const int *E, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partial[i];
    out[0] = ldexp(sqrt(s), *E);
  }
}

// Moves the root factor of sweep 1 (n entries) to the pushed-factor region, dividing it by
// 2^e when its largest entry leaves [2^-32, 2^32] and adding e to E.
// Also writes the factor split into FP32 pairs (hi, lo) for the FP32-storage leaves.
__global__ void __launch_bounds__(256) k_take_root(const double *root, int n, double *keep, float2 *keep32, int *E) {
  __shared__ double red[8];
  const int e = range_exp(block_absmax(root, n, red));
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = ldexp(root[i], -e);
    keep[i] = v;
    const float hi = (float)v;
    keep32[i] = make_float2(hi, (float)(v - (double)hi));
  }
  if (threadIdx.x == 0 && e != 0) *E += e;
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------

namespace {

constexpr int kMaxLev = 10;
constexpr size_t kSmemBudget = 220 * 1024;
constexpr size_t kSmemPair = 110 * 1024;  // two co-resident leaf CTAs per SM

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes, size_t al = 16) {
    off = align_up(off, al);
    const size_t o = off;
    off += bytes;
    return o;
  }
};

struct Tree {
  int G = 2;                  // fan-in (children per node)
  int nlev = 0;               // number of factor levels (0 if a single leaf)
  int count[kMaxLev + 1];     // count[0] = leaves, count[nlev] = 1
  int lpc[kMaxLev + 1];       // leaves per node at each level
  size_t slot_off[kMaxLev];   // slot index offset of the children of level l+1 (children at level l)
  size_t nslots = 0;
  size_t node_off[kMaxLev + 1];  // offset (in nodes) of level l in per-level buffers
  size_t nnodes = 0;
};

Tree make_tree(int P, int G) {
  Tree tr;
  tr.G = G;
  tr.count[0] = P;
  tr.lpc[0] = 1;
  int l = 0;
  while (tr.count[l] > 1 && l < kMaxLev) {
    tr.count[l + 1] = (tr.count[l] + G - 1) / G;
    tr.lpc[l + 1] = tr.lpc[l] * G;
    ++l;
  }
  tr.nlev = l;
  size_t so = 0, no = 0;
  for (int i = 0; i <= tr.nlev; ++i) {
    tr.node_off[i] = no;
    no += tr.count[i];
    if (i < tr.nlev) {
      tr.slot_off[i] = so;
      so += tr.count[i];
    }
  }
  tr.nslots = so;
  tr.nnodes = no;
  return tr;
}

// Leaves of a core whose sweep-1 matrix has `rows` rows and b columns: two per SM while each
// gets at least 16 b rows, else one per SM (short leaves spend their time in per-tile and
// per-reflector overheads and add tree nodes: on the paper's Model 1, I_n = 2000 at rank 50,
// the tuner found one leaf per SM with the largest tiles 16 % faster than 250 leaves); at
// most I.
int leaves_for(int64_t I, int64_t rows, int b, int nsm) {
  int64_t target = 2 * (int64_t)nsm;
  if (rows < target * 16 * (int64_t)std::max(b, 1)) target = nsm;
  target = std::min<int64_t>(target, (int64_t)1 << kMaxLev);  // a binary tree holds 2^kMaxLev
  return (int)std::max<int64_t>(1, std::min<int64_t>(I, target));
}

// a buffer of `elems` elements either carved from shared memory or, when spilled, placed
// at the next free element of the per-leaf global scratch (negative encoded offset)
struct Place {
  Carve c;
  int spill;  // 0: all in shared memory; 1: running factors and carried blocks to the global
              // scratch; 2: also the carried tile block CT (ranks above ~120)
  size_t g = 0;
  int take(size_t bytes, size_t elems, int level) {
    if (level > 0 && spill >= level) {
      const int off = -1 - (int)g;
      g += elems;
      return off;
    }
    return (int)c.take(bytes);
  }
};

template <typename T>
struct SmemS1 {
  int oRr, oTile, oXs, oPs, oRed, oW, oSc, oTau, ldt;
  size_t bytes, gstride;
};

template <typename T>
SmemS1<T> smem_s1(int b, int rho, int cin, int Tt, int CC, int spill = 0, bool stage_p = false) {
  SmemS1<T> m;
  Place pl{Carve(), spill};
  Carve &c = pl.c;
  m.ldt = b + 1;
  m.oRr = pl.take(sizeof(T) * b * b, (size_t)b * b, 1);
  m.oTile = (int)c.take(sizeof(T) * (size_t)Tt * rho * m.ldt);
  m.oXs = (int)c.take(sizeof(T) * (size_t)CC * Tt * b);
  // the pushed factor's staged copy (FP32-storage types only, see k_s1_leaf)
  m.oPs = stage_p && !std::is_same<T, double>::value
              ? pl.take(sizeof(T) * (size_t)rho * cin, (size_t)rho * cin, 1)
              : (int)c.take(16);
  m.oRed = (int)c.take(sizeof(T) * NT);
  m.oW = (int)c.take(sizeof(T) * std::max(b, 1));
  m.oSc = (int)c.take(sizeof(T) * (std::is_same<T, double>::value ? 4 : 2));  // reflector scalars
  m.oTau = (int)c.take(sizeof(T) * b);
  m.bytes = c.off;
  m.gstride = pl.g;
  return m;
}

template <typename T>
struct SmemS2 {
  int oQ, oCT, oCR, oRr, oXs, oPs, oRed, oW, oSc, oTq, oTv, oTs, ldq, ldv;
  size_t bytes, gstride;
};

// mode A/last: b1 = R_n, K1 = K_{n+1}, Lmax = max rows per slice of V(Y_n) (<= K_n)
template <typename T>
SmemS2<T> smem_s2(int mode, int b1, int K1, int Lmax, int Tt, int cin, int CC, int spill = 0) {
  SmemS2<T> m;
  Place pl{Carve(), spill};
  Carve &c = pl.c;
  m.ldq = b1 + 1;
  m.ldv = K1 + 1;
  size_t qrows = mode == 1 ? 0 : (size_t)Tt * K1;
  size_t vrows = (size_t)Tt * (mode == 1 ? 1 : Lmax);
  size_t qbytes = std::max(qrows * m.ldq, mode == 2 ? 0 : vrows * m.ldv) * sizeof(T);
  m.oQ = (int)c.take(qbytes);
  m.oCT = pl.take(sizeof(T) * (mode == 1 ? 1 : qrows * Lmax), mode == 1 ? 1 : qrows * Lmax, 2);
  m.oCR = pl.take(sizeof(T) * (mode == 1 ? 1 : (size_t)b1 * Lmax), mode == 1 ? 1 : (size_t)b1 * Lmax, 1);
  m.oRr = pl.take(sizeof(T) * (size_t)K1 * K1, (size_t)K1 * K1, 1);
  m.oXs = (int)c.take(sizeof(T) * (mode == 1 ? (size_t)CC * Tt : 1));
  m.oPs = pl.take(sizeof(T) * (mode == 1 ? (size_t)K1 * cin : 1), mode == 1 ? (size_t)K1 * cin : 1, 1);
  m.oRed = (int)c.take(sizeof(T) * NT);
  // the grouped apply's W and T store go to the per-leaf global scratch with the other
  // spilled buffers when a core's buffers do not fit in shared memory
  // (FP64 only: the FP32-storage types apply reflector by reflector, see hh_apply_grouped)
  constexpr bool grouped = std::is_same<T, double>::value;
  const size_t nw = (size_t)std::max(std::max(std::max(b1, K1), Lmax), grouped ? NT : 1);
  m.oW = pl.take(sizeof(T) * nw, nw, 1);
  const int nts = grouped ? apply_tstore(std::max(b1, 1), std::max(Lmax, 1)) : 1;
  m.oTs = pl.take(sizeof(T) * nts, (size_t)nts, 1);
  m.oSc = (int)c.take(sizeof(T) * (grouped ? 4 : 2));  // reflector scalars (double-buffered in hh_factor_la)
  m.oTq = (int)c.take(sizeof(T) * std::max(b1, 1));
  m.oTv = (int)c.take(sizeof(T) * K1);
  m.bytes = c.off;
  m.gstride = pl.g;
  return m;
}

template <typename T>
struct SmemOut {
  int oV, oCT, oCR, oRed, oW, oSc, oTau, oTs, ldv;
  size_t bytes, gstride;
};

template <typename T>
SmemOut<T> smem_out(int K1, int Lmax, int Tt, int spill = 0) {
  SmemOut<T> m;
  Place pl{Carve(), spill};
  Carve &c = pl.c;
  m.ldv = K1 + 1;
  m.oV = (int)c.take(sizeof(T) * (size_t)Tt * Lmax * m.ldv);
  m.oCT = pl.take(sizeof(T) * (size_t)Tt * Lmax * K1, (size_t)Tt * Lmax * K1, 2);
  m.oCR = pl.take(sizeof(T) * (size_t)K1 * K1, (size_t)K1 * K1, 1);
  m.oRed = (int)c.take(sizeof(T) * NT);
  constexpr bool grouped = std::is_same<T, double>::value;  // see smem_s2
  const size_t nw = (size_t)std::max(K1, grouped ? NT : 1);
  m.oW = pl.take(sizeof(T) * nw, nw, 1);
  const int nts = grouped ? apply_tstore(std::max(K1, 1), std::max(K1, 1)) : 1;  // Ln <= K1 columns
  m.oTs = pl.take(sizeof(T) * nts, (size_t)nts, 1);
  m.oSc = (int)c.take(sizeof(T) * (grouped ? 4 : 2));
  m.oTau = (int)c.take(sizeof(T) * K1);
  m.bytes = c.off;
  m.gstride = pl.g;
  return m;
}

struct SmemTree {
  int oA, oB, oRed, oW, oSc, oTau, lda, MT, nchunk;
  int w = 0;  // columns of C per CTA (apply layouts)
  size_t bytes;
};

// Shared memory of the tree kernels.  Factor: A = Rr (b x b), B = tile (MT x lda).
// Apply: A = C (b x w), B = V (MT x lda) + CT (MT x w), w = the columns of C one CTA takes.
// MT = tile rows: (G - 1) b (a node's other triangles at once) when that fits, else b,
// else the largest halving of b that fits (a child in chunks); the apply must fit with
// the factor's MT (the slots hold its chunking) and at least kTreeMinCols columns.
constexpr int kTreeMinCols = 8;

static size_t tree_bytes(int b, int MT, int w, SmemTree *m) {
  Carve c;
  const int oA = (int)c.take((size_t)b * std::max(b, w) * sizeof(double));
  const int oB = (int)c.take(((size_t)MT * (b + 1) + (size_t)MT * w) * sizeof(double));
  const int oRed = (int)c.take(sizeof(double) * NT);
  const int oW = (int)c.take(sizeof(double) * std::max(b, w));
  const int oSc = (int)c.take(sizeof(double) * 4);
  const int oTau = (int)c.take(sizeof(double) * b);
  if (m) {
    m->lda = b + 1;
    m->MT = MT;
    m->oA = oA;
    m->oB = oB;
    m->oRed = oRed;
    m->oW = oW;
    m->oSc = oSc;
    m->oTau = oTau;
    m->bytes = c.off;
    m->nchunk = (b + MT - 1) / MT;
    m->w = w;
  }
  return c.off;
}

// factor layout (w = 0: no CT), MT chosen so that the apply also fits with kTreeMinCols
SmemTree smem_tree(int b, int G) {
  int MT = std::max(1, G - 1) * b;
  for (; MT > 1; MT = MT > b ? b : (MT + 1) / 2)
    if (tree_bytes(b, MT, 0, nullptr) <= kSmemBudget &&
        tree_bytes(b, MT, std::min(b, kTreeMinCols), nullptr) <= kSmemBudget)
      break;
  SmemTree m;
  tree_bytes(b, MT, 0, &m);
  return m;
}

// apply layout for the factor's MT: the widest column chunk (<= cmax) that fits
SmemTree smem_tree_apply(int b, int G, int cmax) {
  const SmemTree f = smem_tree(b, G);
  int w = std::max(1, cmax);
  while (w > 1 && tree_bytes(b, f.MT, w, nullptr) > kSmemBudget) --w;
  SmemTree m;
  tree_bytes(b, f.MT, w, &m);
  return m;
}

// Tree fan-in for factors of b columns: 8 children per node (one pass of b reflectors over
// seven interleaved triangles: a 304-leaf tree has 3 levels instead of the 5 of fan-in 4 and
// the 9 of a binary tree, each level a chain of b reflectors) when such a tile fits in
// shared memory, else 4, 3, 2.  Measured on the large-mode workload (b = 32): trees
// 10.9 ms -> 7.9 ms per rounding against fan-in 4.
int tree_fanin(int b) {
  for (int G : {8, 4, 3}) {
    const SmemTree m = smem_tree(b, G);
    if (m.bytes <= kSmemBudget && m.MT >= (G - 1) * b) return G;
  }
  return 2;
}

// shared bytes of k_svd for K columns (ms = ns = K is the largest case); vglobal: the
// rotation accumulator V lives in global memory
size_t smem_svd(int K, bool precond, bool vglobal = false) {
  const size_t w = precond ? svd_w_doubles(K, K) : 0;
  return sizeof(double) * ((size_t)K * K * (vglobal ? 1 : 2) + w + K + SVD_NT / 32 + 1) +
         sizeof(int) * (3 * (size_t)K + 16);
}

struct CorePlan {
  int64_t I = 0;
  int64_t Ig = 0;      // mode size of the whole tensor (I unless sharded)
  int R0 = 1, R1 = 1;  // input ranks
  int K0 = 1, K1 = 1;  // ranks after sweep 1
  int P = 1, Tt = 1;
  int Tt_want = 0;     // tuned tile (0 = heuristic); clamped to what fits
  int spill = 0;  // 1: running factor / carried blocks in global scratch, 2: also the tile block CT
  Tree tree;
  Tree stree;          // sharded: tree over the shards' roots (one leaf per shard)
  size_t refl_off = 0, tau_off = 0, slot_off = 0;  // sweep-1 storage (n >= 1)
  size_t sslot_off = 0;  // sharded: sweep-1 slots of the shard-level tree (n >= 1)
};

TileKey core_key(const CorePlan &c, int prec, int ctx) {
  TileKey k;
  k.prec = prec;
  k.ctx = ctx;
  k.I = c.I;
  k.R0 = c.R0;
  k.R1 = c.R1;
  k.K0 = c.K0;
  k.K1 = c.K1;
  return k;
}

}  // namespace

struct RoundPlan {
  bool keep_q = true;  // store sweep-1 reflectors (rounding); the norm keeps only R
  size_t gscr_elems = 0;  // global scratch for spilled leaf buffers (elements of the compute type)
  size_t off_gscr = 0;
  int N = 0;
  int dtype = TT_F64;
  int nsm = 152;
  int bmax = 1;  // max input rank
  std::vector<CorePlan> core;
  // workspace layout (bytes)
  size_t off_ctl = 0, off_L = 0, off_scal = 0, off_status = 0, off_P = 0, off_P32 = 0;
  size_t off_R = 0, off_C1 = 0, off_C2 = 0, off_slots2 = 0, off_refl2 = 0, off_tau2 = 0, off_part = 0, off_svdV = 0;
  size_t max_nodes = 0, max_slots = 0;
  size_t total = 0;
  int tree_MT[TT_MAX_RANK + 1];
  // sharded rounding: shard-level tree levels (R, and C for the two applies), the
  // V-QR slots of the shard-level tree
  int world = 1, rank = 0;
  size_t off_Rs = 0, off_Cs1 = 0, off_Cs2 = 0, off_sslots2 = 0;
};

// Slab of a sharded tensor: shard `rank` of `world` owns slices
// [leaf_begin(Ig, world, rank), leaf_begin(Ig, world, rank + 1)) of every mode.
struct ShardGeom {
  int world = 1, rank = 0;
  const int64_t *Ig = nullptr;
};

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 152;
  return n;
}

// largest shared-memory footprint of the kernels that core n runs with tile Tt
template <typename T>
static size_t core_smem(const RoundPlan &pl, int n, int Tt, int spill, bool sweep1_only, size_t *gstride) {
  const CorePlan &c = pl.core[n];
  const int N = pl.N, CC = 8;
  size_t mx = 0, g = 0;
  auto acc = [&](size_t bytes, size_t gs) {
    mx = std::max(mx, bytes);
    g = std::max(g, gs);
  };
  if (n >= 1) {
    const SmemS1<T> a = smem_s1<T>(c.R0, c.K1, c.R1, Tt, CC, spill, true);
    acc(a.bytes, a.gstride);
    if (!sweep1_only) {
      if (n < N - 1) {
        const SmemS2<T> b = smem_s2<T>(0, c.R0, c.K1, c.K0, Tt, 1, CC, spill);
        const SmemOut<T> o = smem_out<T>(c.K1, c.K0, Tt, spill);
        acc(b.bytes, b.gstride);
        acc(o.bytes, o.gstride);
      } else {
        const SmemS2<T> b = smem_s2<T>(2, c.R0, c.K1, c.K0, Tt, 1, CC, spill);
        acc(b.bytes, b.gstride);
      }
    }
  } else if (!sweep1_only) {
    const SmemS2<T> b = smem_s2<T>(1, 1, c.K1, 1, Tt, c.R1, CC, spill);
    const SmemOut<T> o = smem_out<T>(c.K1, 1, Tt, spill);
    acc(b.bytes, b.gstride);
    acc(o.bytes, o.gstride);
  }
  if (gstride) *gstride = g;
  return mx;
}

// Tile height (slices per tile) per core: the largest that fits, then shrunk while that
// lets two leaf CTAs share an SM.  Cores whose buffers do not fit even with one slice per
// tile move their running factor and carried block to a per-leaf global scratch.
template <typename T>
static bool choose_tiles(RoundPlan &pl, bool sweep1_only, int ctx) {
  const int N = pl.N;
  pl.gscr_elems = 0;
  for (int n = 0; n < N; ++n) {
    CorePlan &c = pl.core[n];
    if (sweep1_only && n == 0) continue;
    const int64_t per_leaf = (c.I + c.P - 1) / c.P;
    const int maxT = n == 0 ? 512 : 64;
    int best = 0;
    for (int sp = 0; sp < 3 && best == 0; ++sp) {
      c.spill = sp;
      for (int Tt = 1; Tt <= maxT && Tt <= per_leaf; ++Tt) {
        if (n >= 1 && Tt * c.K1 > 512 && Tt > 1) break;
        if (core_smem<T>(pl, n, Tt, c.spill, sweep1_only, nullptr) > kSmemBudget) break;
        best = Tt;
      }
    }
    if (best == 0) return false;
    c.Tt = best;
    if (c.Tt_want > 0) {
      c.Tt = std::min(best, c.Tt_want);
    } else if (ctx == kCtxSolo && c.P <= pl.nsm) {
      // one leaf per SM: the largest tile that fits
      c.Tt = best;
    } else {
      // heuristic: the largest tile that lets two leaves share an SM
      for (int Tt = best; Tt >= 1; --Tt) {
        if (core_smem<T>(pl, n, Tt, c.spill, sweep1_only, nullptr) <= kSmemPair) {
          c.Tt = Tt;
          break;
        }
      }
    }
    size_t g = 0;
    core_smem<T>(pl, n, c.Tt, c.spill, sweep1_only, &g);
    pl.gscr_elems = std::max(pl.gscr_elems, g * (size_t)c.P);
  }
  return true;
}

template <typename T>
static int make_plan(const tt_tensor *x, RoundPlan &pl, bool sweep1_only, int prec, int ctx,
                     const ShardGeom *sg = nullptr) {
  const int N = x->N;
  pl.N = N;
  pl.keep_q = !sweep1_only;
  pl.dtype = x->dtype;
  pl.nsm = device_sm_count();
  pl.core.assign(N, CorePlan());
  pl.bmax = 1;
  for (int n = 0; n < N; ++n) {
    CorePlan &c = pl.core[n];
    c.I = x->I[n];
    c.Ig = sg ? sg->Ig[n] : c.I;
    c.R0 = (int)x->R[n];
    c.R1 = (int)x->R[n + 1];
    pl.bmax = std::max(pl.bmax, std::max(c.R0, c.R1));
  }
  // ranks after the right-to-left sweep: K_n = min(R_n, I_n K_{n+1}), I_n of the whole tensor
  pl.core[N - 1].K1 = 1;
  for (int n = N - 1; n >= 1; --n) {
    CorePlan &c = pl.core[n];
    c.K0 = (int)std::min<int64_t>(c.R0, c.Ig * c.K1);
    pl.core[n - 1].K1 = c.K0;
  }
  pl.core[0].K0 = 1;
  for (int n = 0; n < N; ++n) {
    CorePlan &c = pl.core[n];
    // the core's tall-skinny matrix: H(X_n)^T ((I K_{n+1}) x R_n) in sweep 1, V(X_1) (I x K_2) for core 1
    c.P = n == 0 ? leaves_for(c.I, c.I, c.K1, pl.nsm) : leaves_for(c.I, c.I * c.K1, c.R0, pl.nsm);
    // a batch member shares the GPU with the members on the other streams: at most one
    // leaf per two SMs by default (the batch tuner's usual pick)
    if (ctx == kCtxBatch) c.P = std::min(c.P, std::max(1, pl.nsm / 2));
    TileChoice tc;
    if (tile_choice(core_key(c, prec, ctx), &tc)) {
      if (tc.P > 0) c.P = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)tc.P, c.I, (int64_t)1 << kMaxLev}));
      c.Tt_want = tc.Tt;
    }
    c.tree = make_tree(c.P, std::min(tree_fanin(c.R0), tree_fanin(c.K1)));
    if (sg) c.stree = make_tree(sg->world, c.tree.G);
  }
  if (N > 1 && !choose_tiles<T>(pl, sweep1_only, ctx)) return TT_ERR_UNSUPPORTED;
  // svd and tree shared-memory limits
  for (int n = 0; n + 1 < N && !sweep1_only; ++n)
    if (smem_svd(pl.core[n].K1, false, true) > kSmemBudget) return TT_ERR_UNSUPPORTED;
  for (int n = 1; n < N; ++n)
    if (smem_tree(pl.core[n].R0, pl.core[n].tree.G).bytes > kSmemBudget) return TT_ERR_UNSUPPORTED;
  // workspace layout
  Carve w;
  pl.off_L = w.take(sizeof(int) * (N + 1), 256);
  pl.off_scal = w.take(sizeof(double) * 4, 256);
  pl.off_status = w.take(sizeof(int) * 4, 256);
  pl.off_P = w.take(sizeof(double) * (size_t)pl.bmax * pl.bmax, 256);
  pl.off_P32 = w.take(sizeof(float2) * (size_t)pl.bmax * pl.bmax, 256);
  size_t max_nodes = 1, max_slots = 1, max_refl2 = 1, max_tau2 = 1;
  const size_t B = (size_t)pl.bmax;
  for (int n = 0; n < N; ++n) {
    CorePlan &c = pl.core[n];
    max_nodes = std::max(max_nodes, c.tree.nnodes);
    max_slots = std::max(max_slots, c.tree.nslots);
    if (n >= 1 && pl.keep_q) {
      c.refl_off = w.take(sizeof(T) * (size_t)c.I * c.K1 * c.R0, 256);
      c.tau_off = w.take(sizeof(T) * (size_t)c.I * c.R0, 256);
      const SmemTree st = smem_tree(c.R0, c.tree.G);
      c.slot_off = w.take(sizeof(double) * c.tree.nslots * ((size_t)c.R0 * c.R0 + (size_t)st.nchunk * c.R0), 256);
    }
    if (n < N - 1) {
      max_refl2 = std::max(max_refl2, (size_t)c.I * c.K0 * c.K1);
      max_tau2 = std::max(max_tau2, (size_t)c.I * c.K1);
    }
  }
  pl.max_nodes = max_nodes;
  pl.max_slots = max_slots;
  pl.off_R = w.take(sizeof(double) * max_nodes * B * B, 256);
  pl.off_C1 = w.take(sizeof(double) * max_nodes * B * B, 256);
  pl.off_C2 = w.take(sizeof(double) * max_nodes * B * B, 256);
  if (pl.keep_q) {
    pl.off_slots2 = w.take(sizeof(double) * max_slots * (B * B + B * B), 256);
    pl.off_refl2 = w.take(sizeof(T) * max_refl2, 256);
    pl.off_tau2 = w.take(sizeof(T) * max_tau2, 256);
  }
  if (sg) {
    pl.world = sg->world;
    pl.rank = sg->rank;
    size_t snodes = 1, sslots2 = 1;
    for (int n = 0; n < N; ++n) {
      CorePlan &c = pl.core[n];
      snodes = std::max(snodes, c.stree.nnodes);
      if (n >= 1) {
        const SmemTree st = smem_tree(c.R0, c.stree.G);
        c.sslot_off = w.take(sizeof(double) * c.stree.nslots * ((size_t)c.R0 * c.R0 + (size_t)st.nchunk * c.R0), 256);
      }
      if (n < N - 1) {
        const SmemTree st = smem_tree(c.K1, c.stree.G);
        sslots2 = std::max(sslots2, c.stree.nslots * ((size_t)c.K1 * c.K1 + (size_t)st.nchunk * c.K1));
      }
    }
    pl.off_Rs = w.take(sizeof(double) * snodes * B * B, 256);
    pl.off_Cs1 = w.take(sizeof(double) * snodes * B * B, 256);
    pl.off_Cs2 = w.take(sizeof(double) * snodes * B * B, 256);
    pl.off_sslots2 = w.take(sizeof(double) * sslots2, 256);
  }
  pl.off_part = w.take(sizeof(double) * 4096, 256);
  pl.off_svdV = w.take(sizeof(double) * B * B, 256);
  pl.off_gscr = w.take(sizeof(T) * std::max<size_t>(pl.gscr_elems, 1), 256);
  pl.total = w.off;
  return TT_OK;
}

// compute type of each precision: FP64 -> double, FP32X2 -> df32 (pairs of floats), FP32 -> float
static int plan_for(const tt_tensor *x, int prec, RoundPlan &pl, bool sweep1_only, int ctx = kCtxSolo,
                    const ShardGeom *sg = nullptr) {
  switch (prec) {
    case TT_PREC_FP64: return make_plan<double>(x, pl, sweep1_only, prec, ctx, sg);
    case TT_PREC_FP32X2: return make_plan<df32>(x, pl, sweep1_only, prec, ctx, sg);
    case TT_PREC_FP32: return make_plan<float>(x, pl, sweep1_only, prec, ctx, sg);
    default: return TT_ERR_INVALID_ARG;
  }
}

int tile_classes(const tt_tensor *x, int prec, int ctx, std::vector<TileKey> *keys, std::vector<TileChoice> *heur,
                 std::vector<int64_t> *elems) {
  keys->clear();
  heur->clear();
  elems->clear();
  if (x->N < 2) return TT_OK;
  RoundPlan pl;
  int st = plan_for(x, prec, pl, false, ctx);
  if (st) return st;
  for (const CorePlan &c : pl.core) {
    const TileKey k = core_key(c, prec, ctx);
    const int64_t e = (int64_t)c.R0 * c.I * c.R1;
    size_t i = 0;
    while (i < keys->size() && !((*keys)[i] == k)) ++i;
    if (i == keys->size()) {
      keys->push_back(k);
      heur->push_back(TileChoice{c.P, c.Tt});
      elems->push_back(0);
    }
    (*elems)[i] += e;
  }
  return TT_OK;
}

int round_workspace(const tt_tensor *x, int prec, size_t *bytes, int ctx) {
  RoundPlan pl;
  int st = plan_for(x, prec, pl, false, ctx);
  if (st) return st;
  *bytes = pl.total;
  return TT_OK;
}

#define TT_CUDA(call)                          \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return TT_ERR_CUDA; \
  } while (0)

template <typename K>
static int set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) TT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return TT_OK;
}

// level-by-level tree factorization of the leaf R's in Rbuf level 0; root ends at level nlev
static int tree_factor(const Tree &tr, int b, int64_t I, int rho, const int *rho_dyn, double *Rbase, double *slots,
                       int B, cudaStream_t st) {
  const SmemTree sm = smem_tree(b, tr.G);  // the apply replays this chunking
  int r = set_smem(k_tree_factor, sm.bytes);
  if (r) return r;
  for (int l = 0; l < tr.nlev; ++l) {
    TreeArgs a{};
    a.Rin = Rbase + tr.node_off[l] * B * B;
    a.Rout = Rbase + tr.node_off[l + 1] * B * B;
    a.slots = slots ? slots + tr.slot_off[l] * ((size_t)b * b + (size_t)sm.nchunk * b) : nullptr;
    a.nchild = tr.count[l];
    a.G = tr.G;
    a.b = b;
    a.MT = sm.MT;
    a.nchunk = sm.nchunk;
    a.I = I;
    a.P = tr.count[0];
    a.lpc = tr.lpc[l];
    a.rho = rho;
    a.rho_dyn = rho_dyn;
    a.lda = sm.lda;
    a.oA = sm.oA;
    a.oB = sm.oB;
    a.oRed = sm.oRed;
    a.oW = sm.oW;
    a.oSc = sm.oSc;
    a.oTau = sm.oTau;
    {
      TraceScope ts_(TT_K_TREE_FACTOR, st);
      k_tree_factor<<<tr.count[l + 1], NT, sm.bytes, st>>>(a);
    }
    TT_CUDA(cudaGetLastError());
  }
  return TT_OK;
}

// root-to-leaves application; the root C sits at Cbase level nlev; leaf C's end at level 0
static int tree_apply(const Tree &tr, int b, int64_t I, int rho, const int *rho_dyn, int ncol, const int *ncol_dyn,
                      int cmax, double *Cbase, const double *slots, int B, cudaStream_t st) {
  const int pl_nsm = device_sm_count();
  // the factorization's tile rows (its chunking is in the slots), and the widest column
  // chunk of C one CTA can take next to them
  const SmemTree use = smem_tree_apply(b, tr.G, cmax);
  const int wmax = use.w;
  if (use.bytes > kSmemBudget || tr.G * use.nchunk > 64 || wmax < 1) return TT_ERR_UNSUPPORTED;
  int r = set_smem(k_tree_apply, use.bytes);
  if (r) return r;
  for (int l = tr.nlev - 1; l >= 0; --l) {
    TreeArgs a{};
    a.Cin = Cbase + tr.node_off[l + 1] * B * B;
    a.Cout = Cbase + tr.node_off[l] * B * B;
    a.slots = const_cast<double *>(slots) + tr.slot_off[l] * ((size_t)b * b + (size_t)use.nchunk * b);
    a.nchild = tr.count[l];
    a.G = tr.G;
    a.b = b;
    a.MT = use.MT;
    a.nchunk = use.nchunk;
    a.I = I;
    a.P = tr.count[0];
    a.lpc = tr.lpc[l];
    a.rho = rho;
    a.rho_dyn = rho_dyn;
    a.ncol = ncol;
    a.ncol_dyn = ncol_dyn;
    a.ldc = B;
    a.lda = use.lda;
    a.oA = use.oA;
    a.oB = use.oB;
    a.oRed = use.oRed;
    a.oW = use.oW;
    a.oSc = use.oSc;
    a.oTau = use.oTau;
    // one CTA per node, the columns of C split over more CTAs while the level has fewer
    // nodes than SMs (at least 8 columns each), and always into chunks of at most wmax
    const int ny = std::max((cmax + wmax - 1) / wmax,
                            std::max(1, std::min((pl_nsm + tr.count[l + 1] - 1) / tr.count[l + 1], (cmax + 7) / 8)));
    {
      TraceScope ts_(TT_K_TREE_APPLY, st);
      k_tree_apply<<<dim3(tr.count[l + 1], ny), NT, use.bytes, st>>>(a);
    }
    TT_CUDA(cudaGetLastError());
  }
  return TT_OK;
}

// Launches of the sweep-2 kernels in the instantiation matching the core's spill mode.
template <typename S, typename T>
static int launch_s2_leaf(const S2Args<S, T> &a, int P, size_t bytes, bool spill, cudaStream_t st) {
  auto kern = spill ? k_s2_leaf<S, T, true> : k_s2_leaf<S, T, false>;
  int r = set_smem(kern, bytes);
  if (r) return r;
  {
    TraceScope ts_(TT_K_S2_LEAF, st);
    kern<<<P, NT, bytes, st>>>(a);
  }
  TT_CUDA(cudaGetLastError());
  return TT_OK;
}

template <typename S, typename T>
static int launch_s2_out(const OutArgs<S, T> &a, int P, size_t bytes, bool spill, cudaStream_t st) {
  auto kern = spill ? k_s2_out<S, T, true> : k_s2_out<S, T, false>;
  int r = set_smem(kern, bytes);
  if (r) return r;
  {
    TraceScope ts_(TT_K_S2_OUT, st);
    kern<<<P, NT, bytes, st>>>(a);
  }
  TT_CUDA(cudaGetLastError());
  return TT_OK;
}

// ------------------------------------------------------------------------------------
// sharded rounding: one shard's side of the all-gathers.  Each shard owns a slab of
// every core (the 1 x P x 1 distribution of Sec. 3.1); every tall-skinny QR reduces
// the shards' local roots by an all-gather and a tree over the gathered roots that
// every shard factors alike (the redundant root of the butterfly TSQR, Sec. 3.3.1),
// so applying Q needs no messages (Sec. 3.3.2).  Tree levels keep R nodes b*b apart
// (b x b, leading dimension b) and C nodes b*B apart (b rows, leading dimension B).
// ------------------------------------------------------------------------------------
struct ShardHeader {
  int32_t status;  // the sender's status (0 = fine)
  int32_t seq;     // index of this all-gather within the call
  uint64_t check;  // digest of the call's arguments (first all-gather), else 0
};

class Shard {
 public:
  Shard(const tt_shard *s, int B) : s_(s), B_(B), block_(sizeof(double) * (size_t)B * B) {}
  int seq() const { return seq_; }

  // All-gather of this shard's header and, after the first exchange, of `elems` <= B*B
  // doubles (device src; zeros if null) into dst (device, world runs of `elems` doubles
  // back to back in rank order; skipped if null).  Every payload after the first has the
  // same size (header and B*B doubles).  Returns the status every shard agrees on: the
  // first nonzero in rank order, where a shard out of step or with another digest than
  // shard 0 counts as TT_ERR_INVALID_ARG; TT_ERR_COMM if the callback fails.
  int exchange(const double *src, double *dst, size_t elems, int status, uint64_t check, bool header_only,
               cudaStream_t st) {
    const size_t bytes = sizeof(ShardHeader) + (header_only ? 0 : block_);
    const size_t run = sizeof(double) * elems;
    const int W = s_->world_size;
    send_.assign(bytes, 0);
    recv_.assign(bytes * W, 0);
    ShardHeader h{status, seq_++, check};
    if (!h.status && run > block_) h.status = TT_ERR_INVALID_ARG;
    if (!h.status) {
      // the synchronization also surfaces a fault of the work queued so far
      if (src && !header_only && run &&
          cudaMemcpyAsync(send_.data() + sizeof h, src, run, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        h.status = TT_ERR_CUDA;
      if (cudaStreamSynchronize(st) != cudaSuccess) h.status = TT_ERR_CUDA;
    }
    std::memcpy(send_.data(), &h, sizeof h);
    if (s_->allgather(send_.data(), recv_.data(), bytes, s_->ctx) != 0) return TT_ERR_COMM;
    ShardHeader q0;
    std::memcpy(&q0, recv_.data(), sizeof q0);
    for (int p = 0; p < W; ++p) {
      ShardHeader q;
      std::memcpy(&q, recv_.data() + (size_t)p * bytes, sizeof q);
      if (q.status) return q.status;
      if (q.seq != q0.seq || q.check != q0.check) return TT_ERR_INVALID_ARG;
    }
    if (dst && !header_only && run)
      TT_CUDA(cudaMemcpy2DAsync(dst, run, recv_.data() + sizeof h, bytes, run, W, cudaMemcpyHostToDevice, st));
    return TT_OK;
  }

  // Shard-level factorization: gathers every shard's local root (a b x b node at
  // local_root) as the leaves of c.stree (level 0 of Rs) and factors that tree; *root is
  // its root (the R factor of the whole tall-skinny matrix, the same on every shard).
  int factor(const CorePlan &c, int b, int rho, const int *rho_dyn, const double *local_root, double *Rs,
             double *slots, cudaStream_t st, double **root) {
    int r = exchange(local_root, Rs + c.stree.node_off[0] * (size_t)B_ * B_, (size_t)b * b, 0, 0, false, st);
    if (r) return r;
    r = tree_factor(c.stree, b, c.Ig, rho, rho_dyn, Rs, slots, B_, st);
    if (r) return r;
    *root = Rs + c.stree.node_off[c.stree.nlev] * (size_t)B_ * B_;
    return TT_OK;
  }

  // Shard-level apply: the C at the root of c.stree (in Cs) down to one block per shard;
  // this shard's block becomes the root C of its local tree (local_root_C).  No messages.
  int apply(const CorePlan &c, int b, int rho, const int *rho_dyn, const int *ncol_dyn, int cmax, double *Cs,
            const double *slots, double *local_root_C, cudaStream_t st) {
    int r = tree_apply(c.stree, b, c.Ig, rho, rho_dyn, 0, ncol_dyn, cmax, Cs, slots, B_, st);
    if (r) return r;
    const size_t node = (size_t)b * B_;
    TT_CUDA(cudaMemcpyAsync(local_root_C, Cs + c.stree.node_off[0] * (size_t)B_ * B_ + (size_t)s_->rank * node,
                            sizeof(double) * node, cudaMemcpyDeviceToDevice, st));
    return TT_OK;
  }

 private:
  const tt_shard *s_;
  int B_;
  size_t block_;
  int seq_ = 0;
  std::vector<unsigned char> send_, recv_;
};

// Source of core n of x, or of the Hadamard product of x and xb when xb is given.
template <typename S>
static CoreSrc<S> core_src(const tt_tensor *x, const tt_tensor *xb, int n) {
  CoreSrc<S> c;
  c.X = reinterpret_cast<const S *>(x->cores[n]);
  c.I = x->I[n];
  c.R0 = (int)x->R[n];
  if (xb) {
    c.B = reinterpret_cast<const S *>(xb->cores[n]);
    c.ra0 = (int)x->R[n];
    c.rb0 = (int)xb->R[n];
    c.rb1 = (int)xb->R[n + 1];
    c.R0 = c.ra0 * c.rb0;
  }
  return c;
}

template <typename S, typename T>
static int sweep1(const RoundPlan &pl, const tt_tensor *x, unsigned char *ws, cudaStream_t st, int *E,
                  const tt_tensor *xb = nullptr, Shard *sh = nullptr) {
  const int N = pl.N;
  const int B = pl.bmax;
  double *Rbase = reinterpret_cast<double *>(ws + pl.off_R);
  const double *Pm = nullptr;  // root R of the previous core (device), K_{n+1} x R_{n+1}
  for (int n = N - 1; n >= 1; --n) {
    const CorePlan &c = pl.core[n];
    // FP32-storage types stage the pushed factor only while two leaf CTAs still fit on an SM
    const bool stage = !std::is_same<T, double>::value && !c.spill &&
                       smem_s1<T>(c.R0, c.K1, c.R1, c.Tt, 8, false, true).bytes <= kSmemPair;
    const SmemS1<T> m = smem_s1<T>(c.R0, c.K1, c.R1, c.Tt, 8, c.spill, stage);
    S1Args<S, T> a{};
    a.gscr = reinterpret_cast<T *>(ws + pl.off_gscr);
    a.gstride = m.gstride;
    a.X = core_src<S>(x, xb, n);
    a.g = Geom{c.I, c.P, c.Tt};
    a.b = c.R0;
    a.cin = c.R1;
    a.rho = c.K1;
    a.Pm = Pm;
    a.Pm32 = Pm ? reinterpret_cast<const float2 *>(ws + pl.off_P32) : nullptr;
    a.stage_p = stage ? 1 : 0;
    a.refl = pl.keep_q ? reinterpret_cast<T *>(ws + c.refl_off) : nullptr;
    a.tau = pl.keep_q ? reinterpret_cast<T *>(ws + c.tau_off) : nullptr;
    a.Rleaf = Rbase + c.tree.node_off[0] * B * B;
    a.CC = 8;
    a.oRr = m.oRr;
    a.oTile = m.oTile;
    a.oXs = m.oXs;
    a.oPs = m.oPs;
    a.oRed = m.oRed;
    a.oW = m.oW;
    a.oSc = m.oSc;
    a.oTau = m.oTau;
    a.ldt = m.ldt;
    int r = set_smem(k_s1_leaf<S, T>, m.bytes);
    if (r) return r;
    {
      TraceScope ts_(TT_K_S1_LEAF, st);
      k_s1_leaf<S, T><<<c.P, NT, m.bytes, st>>>(a);
    }
    TT_CUDA(cudaGetLastError());
    r = tree_factor(c.tree, c.R0, c.I, c.K1, nullptr, Rbase,
                    pl.keep_q ? reinterpret_cast<double *>(ws + c.slot_off) : nullptr, B, st);
    if (r) return r;
    // move the root to the dedicated pushed-factor region so that the next core's leaves
    // can overwrite the tree levels
    double *root = Rbase + c.tree.node_off[c.tree.nlev] * B * B;
    if (sh) {
      r = sh->factor(c, c.R0, c.K1, nullptr, root, reinterpret_cast<double *>(ws + pl.off_Rs),
                     reinterpret_cast<double *>(ws + c.sslot_off), st, &root);
      if (r) return r;
    }
    double *keep = reinterpret_cast<double *>(ws + pl.off_P);
    float2 *keep32 = reinterpret_cast<float2 *>(ws + pl.off_P32);
    // root is b x b row-major with K0 valid rows; the push needs K0 x R0 with ld R0 == b
    {
      TraceScope ts_(TT_K_MISC, st);
      k_take_root<<<1, 256, 0, st>>>(root, c.R0 * c.R0, keep, keep32, E);
    }
    TT_CUDA(cudaGetLastError());
    Pm = keep;
  }
  return TT_OK;
}

// Queues a whole rounding on st.  Sync mode (ranks_dev == nullptr): waits and returns the
// ranks in out->R.  Async mode: copies the ranks (N+1 ints) to ranks_dev and the status
// word to status_dev, device side, and returns without a host synchronization.
template <typename S, typename T>
static int run_round(const RoundPlan &pl, const tt_tensor *x, double eps, tt_tensor *out, unsigned char *ws,
                     cudaStream_t st, int *ranks_dev = nullptr, int *status_dev = nullptr,
                     const tt_tensor *xb = nullptr, Shard *sh = nullptr) {
  const int N = pl.N;
  const int B = pl.bmax;
  int *dL = reinterpret_cast<int *>(ws + pl.off_L);
  double *dscal = reinterpret_cast<double *>(ws + pl.off_scal);
  int *dstatus = reinterpret_cast<int *>(ws + pl.off_status);
  // L[0] = L[N] = 1 are fixed; the others are written by the SVD kernels
  {
    TraceScope ts_(TT_K_MISC, st);
    k_init_ctl<<<1, 32, 0, st>>>(dL, N, dstatus);
  }
  TT_CUDA(cudaGetLastError());
  int *dE = dstatus + 2;  // exponent of the sweep-1 rescaling (zeroed above)
  int r = sweep1<S, T>(pl, x, ws, st, dE, xb, sh);
  if (r) return r;
  double *Rbase = reinterpret_cast<double *>(ws + pl.off_R);
  double *C1 = reinterpret_cast<double *>(ws + pl.off_C1);
  double *C2 = reinterpret_cast<double *>(ws + pl.off_C2);
  // sharded: the shard-level trees' R levels and the C levels of their applies
  double *Rs = reinterpret_cast<double *>(ws + pl.off_Rs);
  double *Cs1 = reinterpret_cast<double *>(ws + pl.off_Cs1);
  double *Cs2 = reinterpret_cast<double *>(ws + pl.off_Cs2);
  double *sslots2 = reinterpret_cast<double *>(ws + pl.off_sslots2);
  const double *P1 = reinterpret_cast<const double *>(ws + pl.off_P);  // R_1 pushed into core 0
  double *slots2 = reinterpret_cast<double *>(ws + pl.off_slots2);
  T *refl2 = reinterpret_cast<T *>(ws + pl.off_refl2);
  T *tau2 = reinterpret_cast<T *>(ws + pl.off_tau2);

  for (int n = 0; n + 1 < N; ++n) {
    const CorePlan &c = pl.core[n];
    const int K1 = c.K1;
    // (a) leaf: Y_n slabs and V-QR
    if (n >= 1) {
      // Q_n tree apply: root C at C1 level nlev (written by the previous SVD; sharded: at
      // the shard-level root in Cs1, applied down to this shard's block first)
      if (sh) {
        r = sh->apply(c, c.R0, c.K1, nullptr, dL + n, c.K0, Cs1, reinterpret_cast<double *>(ws + c.sslot_off),
                      C1 + c.tree.node_off[c.tree.nlev] * (size_t)B * B, st);
        if (r) return r;
      }
      r = tree_apply(c.tree, c.R0, c.I, c.K1, nullptr, 0, dL + n, c.K0, C1,
                     reinterpret_cast<double *>(ws + c.slot_off), B, st);
      if (r) return r;
    }
    {
      const int mode = n == 0 ? 1 : 0;
      const SmemS2<T> m = smem_s2<T>(mode, n == 0 ? 1 : c.R0, K1, n == 0 ? 1 : c.K0, c.Tt, c.R1, 8, c.spill);
      S2Args<S, T> a{};
      a.gscr = reinterpret_cast<T *>(ws + pl.off_gscr);
      a.gstride = m.gstride;
      a.mode = mode;
      a.g = Geom{c.I, c.P, c.Tt};
      if (n >= 1) {
        a.qrefl = reinterpret_cast<const T *>(ws + c.refl_off);
        a.qtau = reinterpret_cast<const T *>(ws + c.tau_off);
        a.b1 = c.R0;
        a.Cleaf = C1 + c.tree.node_off[0] * (size_t)B * B;
        a.ldc = B;
        a.Lcur = dL + n;
      } else {
        a.b1 = 1;
        a.X0 = core_src<S>(x, xb, 0);
        a.cin = c.R1;
        a.Pm = N > 1 ? P1 : nullptr;
        a.CC = 8;
      }
      a.K1 = K1;
      a.vrefl = refl2;
      a.vtau = tau2;
      a.Rleaf = Rbase + c.tree.node_off[0] * (size_t)B * B;
      a.oQ = m.oQ;
      a.oCT = m.oCT;
      a.oCR = m.oCR;
      a.oRr = m.oRr;
      a.oXs = m.oXs;
      a.oPs = m.oPs;
      a.oRed = m.oRed;
      a.oW = m.oW;
      a.oTs = m.oTs;
      a.oSc = m.oSc;
      a.oTq = m.oTq;
      a.oTv = m.oTv;
      a.ldq = m.ldq;
      a.ldv = m.ldv;
      r = launch_s2_leaf(a, c.P, m.bytes, c.spill > 0, st);
      if (r) return r;
    }
    // (b) tree of V-QR factors (rows per slice = L[n])
    r = tree_factor(c.tree, K1, c.I, 1, n == 0 ? nullptr : dL + n, Rbase, slots2, B, st);
    if (r) return r;
    double *Rroot = Rbase + c.tree.node_off[c.tree.nlev] * (size_t)B * B;
    if (sh) {
      r = sh->factor(c, K1, 1, n == 0 ? nullptr : dL + n, Rroot, Rs, sslots2, st, &Rroot);
      if (r) return r;
    }
    // (c) SVD of the root, rank choice, U_hat -> C2 root, C_next -> C1 root of core n+1's
    // tree (sharded: the roots of the shard-level trees)
    {
      const CorePlan &cn = pl.core[n + 1];
      SvdArgs a{};
      a.Rroot = Rroot;
      a.K = K1;
      a.In = c.Ig;
      a.Lcur = dL + n;
      a.Lnext = dL + n + 1;
      a.n = n;
      a.N = N;
      a.eps = eps;
      a.scal = dscal;
      a.E = dE;
      a.Uhat = sh ? Cs2 + c.stree.node_off[c.stree.nlev] * (size_t)B * B
                  : C2 + c.tree.node_off[c.tree.nlev] * (size_t)B * B;
      a.Cnext = sh ? Cs1 + cn.stree.node_off[cn.stree.nlev] * (size_t)B * B
                   : C1 + cn.tree.node_off[cn.tree.nlev] * (size_t)B * B;
      a.ldu = B;
      a.status = dstatus;
      const bool vg = smem_svd(K1, false) > kSmemBudget;
      a.Vg = vg ? reinterpret_cast<double *>(ws + pl.off_svdV) : nullptr;
      a.precond = !vg && smem_svd(K1, true) <= kSmemBudget;
      const size_t bytes = smem_svd(K1, a.precond != 0, vg);
      r = set_smem(k_svd, bytes);
      if (r) return r;
      {
        TraceScope ts_(TT_K_SVD, st);
        k_svd<<<1, SVD_NT, bytes, st>>>(a);
      }
      TT_CUDA(cudaGetLastError());
    }
    // (d) U_hat down the V-QR tree (sharded: the shard-level tree first), then the output core
    if (sh) {
      r = sh->apply(c, K1, 1, n == 0 ? nullptr : dL + n, dL + n + 1, K1, Cs2, sslots2,
                    C2 + c.tree.node_off[c.tree.nlev] * (size_t)B * B, st);
      if (r) return r;
    }
    r = tree_apply(c.tree, K1, c.I, 1, n == 0 ? nullptr : dL + n, 0, dL + n + 1, K1, C2, slots2, B, st);
    if (r) return r;
    {
      const SmemOut<T> m = smem_out<T>(K1, n == 0 ? 1 : c.K0, c.Tt, c.spill);
      OutArgs<S, T> a{};
      a.gscr = reinterpret_cast<T *>(ws + pl.off_gscr);
      a.gstride = m.gstride;
      a.g = Geom{c.I, c.P, c.Tt};
      a.vrefl = refl2;
      a.vtau = tau2;
      a.K1 = K1;
      a.Lcur = dL + n;
      a.Lnext = dL + n + 1;
      a.Uleaf = C2 + c.tree.node_off[0] * (size_t)B * B;
      a.ldc = B;
      a.out = reinterpret_cast<S *>(out->cores[n]);
      a.E = dE;
      a.n = n;
      a.N = N;
      a.oV = m.oV;
      a.oCT = m.oCT;
      a.oCR = m.oCR;
      a.oRed = m.oRed;
      a.oW = m.oW;
      a.oTs = m.oTs;
      a.oSc = m.oSc;
      a.oTau = m.oTau;
      a.ldv = m.ldv;
      r = launch_s2_out(a, c.P, m.bytes, c.spill > 0, st);
      if (r) return r;
    }
  }
  // last core: S_{N-2} x_1 Q_{N-1}
  {
    const CorePlan &c = pl.core[N - 1];
    if (sh) {
      r = sh->apply(c, c.R0, c.K1, nullptr, dL + N - 1, c.K0, Cs1, reinterpret_cast<double *>(ws + c.sslot_off),
                    C1 + c.tree.node_off[c.tree.nlev] * (size_t)B * B, st);
      if (r) return r;
    }
    r = tree_apply(c.tree, c.R0, c.I, c.K1, nullptr, 0, dL + N - 1, c.K0, C1,
                   reinterpret_cast<double *>(ws + c.slot_off), B, st);
    if (r) return r;
    const SmemS2<T> m = smem_s2<T>(2, c.R0, 1, c.K0, c.Tt, 1, 8, c.spill);
    S2Args<S, T> a{};
    a.gscr = reinterpret_cast<T *>(ws + pl.off_gscr);
    a.gstride = m.gstride;
    a.mode = 2;
    a.g = Geom{c.I, c.P, c.Tt};
    a.qrefl = reinterpret_cast<const T *>(ws + c.refl_off);
    a.qtau = reinterpret_cast<const T *>(ws + c.tau_off);
    a.b1 = c.R0;
    a.K1 = 1;
    a.Cleaf = C1 + c.tree.node_off[0] * (size_t)B * B;
    a.ldc = B;
    a.Lcur = dL + N - 1;
    a.out = reinterpret_cast<S *>(out->cores[N - 1]);
    a.E = dE;
    a.n = N - 1;
    a.N = N;
    a.oQ = m.oQ;
    a.oCT = m.oCT;
    a.oCR = m.oCR;
    a.oRr = m.oRr;
    a.oXs = m.oXs;
    a.oPs = m.oPs;
    a.oRed = m.oRed;
    a.oW = m.oW;
    a.oTs = m.oTs;
    a.oSc = m.oSc;
    a.oTq = m.oTq;
    a.oTv = m.oTv;
    a.ldq = m.ldq;
    a.ldv = m.ldv;
    r = launch_s2_leaf(a, c.P, m.bytes, c.spill > 0, st);
    if (r) return r;
  }
  if (ranks_dev) {
    TT_CUDA(cudaMemcpyAsync(ranks_dev, dL, sizeof(int) * (N + 1), cudaMemcpyDeviceToDevice, st));
    TT_CUDA(cudaMemcpyAsync(status_dev, dstatus, sizeof(int), cudaMemcpyDeviceToDevice, st));
    return TT_OK;
  }
  // ranks and status back to the host
  std::vector<int> L(N + 1);
  int status[4];
  TT_CUDA(cudaMemcpyAsync(L.data(), dL, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost, st));
  TT_CUDA(cudaMemcpyAsync(status, dstatus, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  TT_CUDA(cudaStreamSynchronize(st));
  if (sh) {
    // every shard returns the same status
    r = sh->exchange(nullptr, nullptr, 0, status[0], 0, false, st);
    if (r) return r;
  }
  if (status[0]) return status[0];
  for (int n = 0; n <= N; ++n) out->R[n] = L[n];
  return TT_OK;
}

__global__ void k_ranks_one(int *ranks, int *status) {
  if (threadIdx.x < 2) ranks[threadIdx.x] = 1;
  if (threadIdx.x == 0) status[0] = 0;
}

int round_enqueue(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes,
                  cudaStream_t st, int *ranks_dev, int *status_dev, int ctx) {
  if (x->N == 1) {
    const size_t es = x->dtype == TT_F64 ? 8 : 4;
    TT_CUDA(cudaMemcpyAsync(out->cores[0], x->cores[0], es * (size_t)x->I[0], cudaMemcpyDefault, st));
    if (ranks_dev) {
      TraceScope ts_(TT_K_MISC, st);
      k_ranks_one<<<1, 32, 0, st>>>(ranks_dev, status_dev);
      TT_CUDA(cudaGetLastError());
      return TT_OK;
    }
    TT_CUDA(cudaStreamSynchronize(st));
    out->R[0] = out->R[1] = 1;
    return TT_OK;
  }
  RoundPlan pl;
  int r = plan_for(x, prec, pl, false, ctx);
  if (r) return r;
  if (!ws || ws_bytes < pl.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return TT_ERR_WORKSPACE;
  unsigned char *w = reinterpret_cast<unsigned char *>(ws);
  switch (prec) {
    case TT_PREC_FP64: return run_round<double, double>(pl, x, eps, out, w, st, ranks_dev, status_dev);
    case TT_PREC_FP32X2: return run_round<float, df32>(pl, x, eps, out, w, st, ranks_dev, status_dev);
    default: return run_round<float, float>(pl, x, eps, out, w, st, ranks_dev, status_dev);
  }
}

int round_run(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st) {
  return round_enqueue(x, eps, prec, out, ws, ws_bytes, st, nullptr, nullptr);
}

int round_sharded_workspace(const tt_tensor *x, int prec, int world, int rank, const int64_t *Ig, size_t *bytes) {
  if (x->N == 1) {
    *bytes = 0;
    return TT_OK;
  }
  ShardGeom g{world, rank, Ig};
  RoundPlan pl;
  int r = plan_for(x, prec, pl, false, kCtxSolo, &g);
  if (r) return r;
  *bytes = pl.total;
  return TT_OK;
}

// One shard's part of a sharded rounding.  local_status carries this shard's argument
// checks (made by the caller) and check the digest of the arguments all shards must share.
// Exchanges: one header-only handshake; if every shard is fine, exactly 2N - 1 more (one
// per tall-skinny QR, one for the final status), made even after a failure so that the
// shards stay in step.
int round_sharded_run(const tt_tensor *x, double eps, int prec, const tt_shard *shard, int local_status,
                      uint64_t check, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st) {
  RoundPlan pl;
  int B = 1;
  if (!local_status) {
    for (int n = 0; n <= x->N; ++n) B = std::max<int>(B, (int)x->R[n]);
    if (x->N > 1) {
      ShardGeom g{shard->world_size, shard->rank, shard->I_global};
      local_status = plan_for(x, prec, pl, false, kCtxSolo, &g);
      if (!local_status && (!ws || ws_bytes < pl.total || (reinterpret_cast<uintptr_t>(ws) & 255)))
        local_status = TT_ERR_WORKSPACE;
    }
  }
  Shard sh(shard, B);
  int r = sh.exchange(nullptr, nullptr, 0, local_status, check, true, st);
  if (r) return r;  // every shard stops here alike
  const int N = x->N;
  if (N == 1) {
    const size_t es = x->dtype == TT_F64 ? 8 : 4;
    r = cudaMemcpyAsync(out->cores[0], x->cores[0], es * (size_t)x->I[0], cudaMemcpyDefault, st) == cudaSuccess
            ? TT_OK
            : TT_ERR_CUDA;
    const int f = sh.exchange(nullptr, nullptr, 0, r, 0, false, st);
    if (f) return f;
    out->R[0] = out->R[1] = 1;
    return TT_OK;
  }
  unsigned char *w = reinterpret_cast<unsigned char *>(ws);
  switch (prec) {
    case TT_PREC_FP64: r = run_round<double, double>(pl, x, eps, out, w, st, nullptr, nullptr, nullptr, &sh); break;
    case TT_PREC_FP32X2: r = run_round<float, df32>(pl, x, eps, out, w, st, nullptr, nullptr, nullptr, &sh); break;
    default: r = run_round<float, float>(pl, x, eps, out, w, st, nullptr, nullptr, nullptr, &sh); break;
  }
  // after a failure the remaining all-gathers still run, carrying the status
  while (sh.seq() < 2 * N) {
    const int f = sh.exchange(nullptr, nullptr, 0, r ? r : TT_ERR_INVALID_ARG, 0, false, st);
    if (!r) r = f;
  }
  return r;
}

// Rounding of the Hadamard product z = a o b (shape of the product in z) without forming
// it: the leaf kernels read the entries of a and b (see CoreSrc); ranks to out->R.
int round_hadamard_run(const tt_tensor *a, const tt_tensor *b, const tt_tensor *z, double eps, int prec,
                       tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st) {
  RoundPlan pl;
  int r = plan_for(z, prec, pl, false, kCtxSolo);
  if (r) return r;
  if (!ws || ws_bytes < pl.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return TT_ERR_WORKSPACE;
  unsigned char *w = reinterpret_cast<unsigned char *>(ws);
  switch (prec) {
    case TT_PREC_FP64: return run_round<double, double>(pl, a, eps, out, w, st, nullptr, nullptr, b);
    case TT_PREC_FP32X2: return run_round<float, df32>(pl, a, eps, out, w, st, nullptr, nullptr, b);
    default: return run_round<float, float>(pl, a, eps, out, w, st, nullptr, nullptr, b);
  }
}

static int norm_prec(const tt_tensor *x) { return x->dtype == TT_F64 ? TT_PREC_FP64 : TT_PREC_FP32X2; }

int norm_workspace(const tt_tensor *x, size_t *bytes) {
  RoundPlan pl;
  int st = plan_for(x, norm_prec(x), pl, true);
  if (st) return st;
  *bytes = pl.total;
  return TT_OK;
}

template <typename S, typename T>
static int run_norm(const RoundPlan &pl, const tt_tensor *x, double *result, unsigned char *ws, cudaStream_t st) {
  const int N = pl.N;
  int *dE = reinterpret_cast<int *>(ws + pl.off_status) + 2;
  TT_CUDA(cudaMemsetAsync(dE, 0, sizeof(int), st));
  int r = N > 1 ? sweep1<S, T>(pl, x, ws, st, dE) : TT_OK;
  if (r) return r;
  const CorePlan &c0 = pl.core[0];
  double *part = reinterpret_cast<double *>(ws + pl.off_part);
  double *res = reinterpret_cast<double *>(ws + pl.off_scal);
  const double *Pm = N > 1 ? reinterpret_cast<const double *>(ws + pl.off_P) : nullptr;
  const int K = N > 1 ? c0.K1 : 1;
  const int cin = N > 1 ? c0.R1 : 1;
  const int64_t total = c0.I * K;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (total + NT - 1) / NT));
  {
    TraceScope ts_(TT_K_MISC, st);
    k_push_sumsq<S><<<blocks, NT, 0, st>>>(reinterpret_cast<const S *>(x->cores[0]), c0.I, cin, K, Pm, part);
  }
  TT_CUDA(cudaGetLastError());
  {
    TraceScope ts_(TT_K_MISC, st);
    k_sum_sqrt<<<1, 32, 0, st>>>(part, blocks, dE, res);
  }
  TT_CUDA(cudaGetLastError());
  TT_CUDA(cudaMemcpyAsync(result, res, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CUDA(cudaStreamSynchronize(st));
  return TT_OK;
}

// Right-orthonormalization with explicit factors (Alg. 5: TSQR of every H(X_n)^T, then
// TSQR-Apply-Q of the identity to form the orthonormal factor, R pushed into core n-1).
// Sweep 1 of the rounding leaves every core's reflectors stored; each core n >= 1 then
// gets Q_n [I; 0] through its tree and leaves (k_s2_leaf in the explicit-factor mode),
// and core 0 receives the pushed root factor.  Ranks K_n = min(R_n, I_n K_{n+1}) follow
// from the shapes, so nothing waits on the device.
template <typename S, typename T>
static int run_orth(const RoundPlan &pl, const tt_tensor *x, tt_tensor *out, unsigned char *ws, cudaStream_t st) {
  const int N = pl.N;
  const int B = pl.bmax;
  int *dL = reinterpret_cast<int *>(ws + pl.off_L);
  int *dstatus = reinterpret_cast<int *>(ws + pl.off_status);
  {
    TraceScope ts_(TT_K_MISC, st);
    k_init_ctl<<<1, 32, 0, st>>>(dL, N, dstatus);
  }
  TT_CUDA(cudaGetLastError());
  int *dE = dstatus + 2;
  int r = sweep1<S, T>(pl, x, ws, st, dE);
  if (r) return r;
  double *C1 = reinterpret_cast<double *>(ws + pl.off_C1);
  for (int n = 1; n < N; ++n) {
    const CorePlan &c = pl.core[n];
    {
      TraceScope ts_(TT_K_MISC, st);
      k_set_int<<<1, 32, 0, st>>>(dL + n, c.K0);
      k_eye<<<std::max(1, (c.K0 * c.K0 + 255) / 256), 256, 0, st>>>(C1 + c.tree.node_off[c.tree.nlev] * (size_t)B * B,
                                                                     c.K0, B);
    }
    TT_CUDA(cudaGetLastError());
    r = tree_apply(c.tree, c.R0, c.I, c.K1, nullptr, c.K0, nullptr, c.K0, C1,
                   reinterpret_cast<double *>(ws + c.slot_off), B, st);
    if (r) return r;
    const SmemS2<T> m = smem_s2<T>(2, c.R0, c.K1, c.K0, c.Tt, 1, 8, c.spill);
    S2Args<S, T> a{};
    a.gscr = reinterpret_cast<T *>(ws + pl.off_gscr);
    a.gstride = m.gstride;
    a.mode = 3;
    a.g = Geom{c.I, c.P, c.Tt};
    a.qrefl = reinterpret_cast<const T *>(ws + c.refl_off);
    a.qtau = reinterpret_cast<const T *>(ws + c.tau_off);
    a.b1 = c.R0;
    a.K1 = c.K1;
    a.Cleaf = C1 + c.tree.node_off[0] * (size_t)B * B;
    a.ldc = B;
    a.Lcur = dL + n;
    a.out = reinterpret_cast<S *>(out->cores[n]);
    a.E = dE;
    a.n = n;
    a.N = N;
    a.oQ = m.oQ;
    a.oCT = m.oCT;
    a.oCR = m.oCR;
    a.oRr = m.oRr;
    a.oXs = m.oXs;
    a.oPs = m.oPs;
    a.oRed = m.oRed;
    a.oW = m.oW;
    a.oTs = m.oTs;
    a.oSc = m.oSc;
    a.oTq = m.oTq;
    a.oTv = m.oTv;
    a.ldq = m.ldq;
    a.ldv = m.ldv;
    r = launch_s2_leaf(a, c.P, m.bytes, c.spill > 0, st);
    if (r) return r;
  }
  // core 0: X_0 x_3 R_1 (the root factor of core 1, kept at off_P), times 2^E
  {
    const CorePlan &c0 = pl.core[0];
    const int64_t total = c0.I * c0.K1;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (total + NT - 1) / NT));
    TraceScope ts_(TT_K_MISC, st);
    k_push_out<S><<<blocks, NT, 0, st>>>(reinterpret_cast<const S *>(x->cores[0]), c0.I, c0.R1, c0.K1,
                                          reinterpret_cast<const double *>(ws + pl.off_P), dE,
                                          reinterpret_cast<S *>(out->cores[0]));
  }
  TT_CUDA(cudaGetLastError());
  out->R[0] = 1;
  for (int n = 1; n < N; ++n) out->R[n] = pl.core[n].K0;
  out->R[N] = 1;
  return TT_OK;
}

int orth_workspace(const tt_tensor *x, int prec, size_t *bytes) {
  if (x->N == 1) {
    *bytes = 0;
    return TT_OK;
  }
  return round_workspace(x, prec, bytes);
}

int orth_enqueue(const tt_tensor *x, int prec, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st) {
  if (x->N == 1) {
    const size_t es = x->dtype == TT_F64 ? 8 : 4;
    TT_CUDA(cudaMemcpyAsync(out->cores[0], x->cores[0], es * (size_t)x->I[0], cudaMemcpyDefault, st));
    out->R[0] = out->R[1] = 1;
    return TT_OK;
  }
  RoundPlan pl;
  int r = plan_for(x, prec, pl, false);
  if (r) return r;
  if (!ws || ws_bytes < pl.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return TT_ERR_WORKSPACE;
  unsigned char *w = reinterpret_cast<unsigned char *>(ws);
  switch (prec) {
    case TT_PREC_FP64: return run_orth<double, double>(pl, x, out, w, st);
    case TT_PREC_FP32X2: return run_orth<float, df32>(pl, x, out, w, st);
    default: return run_orth<float, float>(pl, x, out, w, st);
  }
}

int norm_run(const tt_tensor *x, double *result, void *ws, size_t ws_bytes, cudaStream_t st) {
  RoundPlan pl;
  int r = plan_for(x, norm_prec(x), pl, true);
  if (r) return r;
  if (!ws || ws_bytes < pl.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return TT_ERR_WORKSPACE;
  unsigned char *w = reinterpret_cast<unsigned char *>(ws);
  return x->dtype == TT_F64 ? run_norm<double, double>(pl, x, result, w, st)
                            : run_norm<float, df32>(pl, x, result, w, st);
}

}  // namespace ttgb
