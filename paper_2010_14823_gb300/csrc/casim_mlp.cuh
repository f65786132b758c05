// Warm-rain surrogate network: 12 -> 256 -> 256 -> 256 -> 4, tanh hidden
// layers, BF16 weights and GEMM operands, FP32 accumulation on the tensor
// cores.  Training (forward, backward, Adam) and inference run on the
// kernels below; the step takes the network's rates where its inputs lie in
// the box spanned by the training data and the scheme's rates elsewhere.
#pragma once

#include <cuda_bf16.h>

#include "casim_device.cuh"
#include "casim_batch.cuh"

namespace casim_dev {

constexpr int kNin = 12, kNinPad = 16, kNh = 256, kNout = 4, kNoutPad = 16;
constexpr int kNParam = kNin * kNh + kNh + 2 * (kNh * kNh + kNh) + kNh * kNout + kNout;
// offsets of the layers in the flat parameter vector (oracle order)
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kNin * kNh, kOffW2 = kOffB1 + kNh, kOffB2 = kOffW2 + kNh * kNh,
              kOffW3 = kOffB2 + kNh, kOffB3 = kOffW3 + kNh * kNh, kOffW4 = kOffB3 + kNh,
              kOffB4 = kOffW4 + kNh * kNout;

// ------------------------------------------------------------ tensor-core GEMM
// C[m][n] = sum_k A(m, k) B(n, k) with A(m, k) = A[m*sam + k*sak] and
// B(n, k) = B[n*sbn + k*sbk] (BF16), FP32 accumulation by mma.sync
// m16n8k16.  Tiles of 64x64 over a 2x2 arrangement of warps; operands are
// gathered with arbitrary strides into k-contiguous shared-memory tiles, so
// one kernel serves the forward pass (W^T), the data gradient (W) and the
// weight gradient (both operands transposed).  The epilogue receives
// (m, n, acc) for m < M, n < N.
struct GemmArgs {
  const __nv_bfloat16 *A;
  long long sam, sak;
  const __nv_bfloat16 *B;
  long long sbn, sbk;
  int M, N, K;
  int kchunk;            // split K: block z sums k in [z kchunk, (z+1) kchunk)
};

constexpr int kGBM = 64, kGBN = 64, kGBK = 32, kGPad = 8;

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <class Epi>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g, const Epi epi) {
  __shared__ __align__(16) __nv_bfloat16 As[kGBM][kGBK + kGPad];
  __shared__ __align__(16) __nv_bfloat16 Bs[kGBN][kGBK + kGPad];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = blockIdx.y * kGBM, n0 = blockIdx.x * kGBN;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  const int kb = blockIdx.z * g.kchunk, ke = min(g.K, kb + g.kchunk);
  // gather order: consecutive threads along the operand's unit-stride index
  const bool a_rows = g.sam == 1 && g.sak != 1, b_rows = g.sbn == 1 && g.sbk != 1;
  for (int k0 = kb; k0 < ke; k0 += kGBK) {
#pragma unroll 4
    for (int i = tid; i < kGBM * kGBK; i += 128) {
      const int r = a_rows ? i % kGBM : i / kGBK, kk = a_rows ? i / kGBM : i % kGBK;
      const int m = m0 + r, k = k0 + kk;
      As[r][kk] = (m < g.M && k < ke) ? g.A[(long long)m * g.sam + (long long)k * g.sak] : zero;
    }
#pragma unroll 4
    for (int i = tid; i < kGBN * kGBK; i += 128) {
      const int r = b_rows ? i % kGBN : i / kGBK, kk = b_rows ? i / kGBN : i % kGBK;
      const int n = n0 + r, k = k0 + kk;
      Bs[r][kk] = (n < g.N && k < ke) ? g.B[(long long)n * g.sbn + (long long)k * g.sbk] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kGBK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16 + gq;
        af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 2 * tq]);
        af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 2 * tq]);
        af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 2 * tq + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = wn * 32 + j * 8 + gq;
        bf[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[r][ks + 2 * tq]);
        bf[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[r][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm * 32 + i * 16 + gq + (r >> 1) * 8;
        const int n = n0 + wn * 32 + j * 8 + 2 * tq + (r & 1);
        if (m < g.M && n < g.N) epi(m, n, acc[i][j][r]);
      }
}

// Epilogues receive (m, n, acc) for m < M, n < N.  One with kLoad = true
// also reads a value per element (load(m, n)); the tensor-core GEMM issues
// those reads for a block of rows before it applies the epilogue
// (apply(m, n, acc, loaded)), so their latencies overlap.

// hidden layer: a = tanh(acc + b); keeps a (FP32, for the backward pass) and
// its BF16 copy (the next layer's input)
struct EpiHidden {
  static constexpr bool kLoad = false;
  const float *bias;
  float *a;              // [M][ld] or null
  __nv_bfloat16 *h;      // [M][ld]
  int ld;
  __device__ __forceinline__ void operator()(int m, int n, float acc) const {
    const float v = tanhf(acc + bias[n]);
    if (a) a[(long long)m * ld + n] = v;
    h[(long long)m * ld + n] = __float2bfloat16(v);
  }
};

// output layer: y = acc + b
struct EpiOut {
  static constexpr bool kLoad = false;
  const float *bias;
  float *y;              // [M][ld]
  int ld;
  __device__ __forceinline__ void operator()(int m, int n, float acc) const { y[(long long)m * ld + n] = acc + bias[n]; }
};

// weight gradient: g[m][n] = acc
struct EpiStore {
  static constexpr bool kLoad = false;
  float *c;
  int ld;
  __device__ __forceinline__ void operator()(int m, int n, float acc) const { c[(long long)m * ld + n] = acc; }
};

// split-K partial sums: ws[z][m][n] for block z
struct EpiPartial {
  static constexpr bool kLoad = false;
  float *ws;
  int ld;
  long long zstride;
  __device__ __forceinline__ void operator()(int m, int n, float acc) const {
    ws[blockIdx.z * zstride + (long long)m * ld + n] = acc;
  }
};

// out[i] = sum over z (in order) of ws[z][i]: deterministic split-K reduction
__global__ void k_splitk_sum(const float *ws, int nsplit, long long len, float *out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= len) return;
  float s = 0.f;
  for (int z = 0; z < nsplit; ++z) s += ws[z * len + i];
  out[i] = s;
}

// data gradient through tanh: dz = acc (1 - a^2); FP32 for the bias sums,
// BF16 for the next GEMMs
struct EpiBackTanh {
  static constexpr bool kLoad = true;
  const float *a;        // [M][ld] activations of the layer below
  float *dz;
  __nv_bfloat16 *dzb;
  int ld;
  __device__ __forceinline__ float load(int m, int n) const { return __ldg(a + (long long)m * ld + n); }
  __device__ __forceinline__ void apply(int m, int n, float acc, float av) const {
    const long long i = (long long)m * ld + n;
    const float v = acc * (1.f - av * av);
    dz[i] = v;
    dzb[i] = __float2bfloat16(v);
  }
  __device__ __forceinline__ void operator()(int m, int n, float acc) const { apply(m, n, acc, load(m, n)); }
};

// ---------------------------------------------------------- elementwise kernels
// master FP32 parameters -> BF16 weight copies in both layouts:
//   Wt[l]: [N][K] (K padded with zeros) for the forward GEMM,
//   Wk[l]: [K][Npad] for the data gradient.
struct MlpBf16 {
  __nv_bfloat16 *w1t, *w2t, *w3t, *w4t;   // [256][16], [256][256], [256][256], [16][256]
  __nv_bfloat16 *w2k, *w3k, *w4k;         // [256][256], [256][256], [256][16]
};

__global__ void k_mlp_cast(const float *theta, MlpBf16 w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  if (i < kNh * kNinPad) {   // w1t[n][k]
    const int n = i / kNinPad, k = i % kNinPad;
    w.w1t[i] = k < kNin ? __float2bfloat16(theta[kOffW1 + k * kNh + n]) : z;
  }
  if (i < kNh * kNh) {
    const int n = i / kNh, k = i % kNh;   // t-layout index i = n*256 + k
    w.w2t[i] = __float2bfloat16(theta[kOffW2 + k * kNh + n]);
    w.w3t[i] = __float2bfloat16(theta[kOffW3 + k * kNh + n]);
    w.w2k[i] = __float2bfloat16(theta[kOffW2 + i]);   // natural [k][n]
    w.w3k[i] = __float2bfloat16(theta[kOffW3 + i]);
  }
  if (i < kNoutPad * kNh) {  // w4t[n][k], n < 16 (rows >= 4 zero)
    const int n = i / kNh, k = i % kNh;
    w.w4t[i] = n < kNout ? __float2bfloat16(theta[kOffW4 + k * kNout + n]) : z;
  }
  if (i < kNh * kNoutPad) {  // w4k[k][n]
    const int k = i / kNoutPad, n = i % kNoutPad;
    w.w4k[i] = n < kNout ? __float2bfloat16(theta[kOffW4 + k * kNout + n]) : z;
  }
}

// FP32 inputs [n][12] -> BF16 [n][16] (zero padded)
__global__ void k_mlp_inputs(const float *X, int n, __nv_bfloat16 *h0) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * kNinPad) return;
  const long long r = i / kNinPad;
  const int k = (int)(i % kNinPad);
  h0[i] = __float2bfloat16(k < kNin ? X[r * kNin + k] : 0.f);
}

// masked squared error: loss += sum (y - t)^2 m / cnt; dz = 2 (y - t) m / cnt
// (FP32 [n][4] and BF16 [n][16], columns >= 4 zero)
__global__ void k_mlp_loss(const float *Y, const float *T, const float *Mk, int n, const float *cnt, double *loss,
                           float *dz, __nv_bfloat16 *dzb) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double part = 0.0;
  if (i < (long long)n * kNoutPad) {
    const long long r = i / kNoutPad;
    const int c = (int)(i % kNoutPad);
    float g = 0.f;
    if (c < kNout) {
      const float inv = 1.f / fmaxf(*cnt, 1.f);
      const float d = (Y[r * kNout + c] - T[r * kNout + c]) * Mk[r * kNout + c];
      part = (double)d * d * inv;
      g = 2.f * d * inv;
      dz[r * kNout + c] = g;
    }
    dzb[i] = __float2bfloat16(g);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(loss, part);
}

__global__ void k_sum(const float *x, long long n, float *out) {
  float part = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    part += x[i];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, part);
}

// bias gradient: column sums of dz [n][ld] (first `cols` columns).  Block
// (32, 32) of grid (column blocks, row chunks): lane x is a column
// (coalesced rows), y a row phase within chunk blockIdx.y; the 32 phase sums
// are added in a fixed order into part[chunk][c]; k_colsum_fin adds the
// chunks in order into g (deterministic).
constexpr int kColsumY = 32, kColsumChunks = 16;
__global__ void __launch_bounds__(32 * kColsumY) k_colsum(const float *dz, int n, int ld, int cols, float *part_out) {
  __shared__ float s_part[kColsumY][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int per = (n + gridDim.y - 1) / gridDim.y, r0 = blockIdx.y * per, r1 = min(n, r0 + per);
  float part = 0.f;
  if (c < cols)
    for (int r = r0 + threadIdx.y; r < r1; r += kColsumY) part += dz[(long long)r * ld + c];
  s_part[threadIdx.y][threadIdx.x] = part;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    float s = 0.f;
    for (int y = 0; y < kColsumY; ++y) s += s_part[y][threadIdx.x];
    part_out[(long long)blockIdx.y * cols + c] = s;
  }
}
__global__ void k_colsum_fin(const float *part, int chunks, int cols, float *g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int y = 0; y < chunks; ++y) s += part[(long long)y * cols + c];
  g[c] = s;
}

// Adam on the flat FP32 parameters
__global__ void k_adam(float *theta, const float *grad, float *m1, float *m2, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float b = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = b;
  theta[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// counter-based mini-batch sampling: row r of batch `step` is
// hash(seed, step, r) mod n (splitmix64 finaliser)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// gather a standardised mini-batch from the raw data
__global__ void k_mlp_batch(const float *X, const float *Y, const float *Mk, long long n, unsigned long long seed,
                            long long step, int B, const float *norm, float *Xn, float *Tn, float *Mb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  const long long src = (long long)(mix64(seed ^ mix64((unsigned long long)step * 0x100000001b3ull + r)) % (unsigned long long)n);
  const float *mu = norm, *sd = norm + kNin, *muy = norm + 2 * kNin, *sdy = norm + 2 * kNin + kNout;
#pragma unroll
  for (int k = 0; k < kNin; ++k) Xn[(long long)r * kNin + k] = (X[src * kNin + k] - mu[k]) / sd[k];
#pragma unroll
  for (int c = 0; c < kNout; ++c) {
    const float m = Mk[src * kNout + c];
    Mb[(long long)r * kNout + c] = m;
    Tn[(long long)r * kNout + c] = m > 0.f ? (Y[src * kNout + c] - muy[c]) / sdy[c] : 0.f;
  }
}

// per-feature mean and standard deviation, per-target (masked) mean and
// standard deviation, per-feature min and max (the box of the training data)
__global__ void k_mlp_stats(const float *X, const float *Y, const float *Mk, long long n, double *acc) {
  // acc: [12 sum][12 sumsq][4 sum][4 sumsq][4 count] then min/max as ordered ints elsewhere
  double s[kNin] = {0}, q[kNin] = {0}, sy[kNout] = {0}, qy[kNout] = {0}, cy[kNout] = {0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < kNin; ++k) {
      const double v = X[i * kNin + k];
      s[k] += v;
      q[k] += v * v;
    }
#pragma unroll
    for (int c = 0; c < kNout; ++c)
      if (Mk[i * kNout + c] > 0.f) {
        const double v = Y[i * kNout + c];
        sy[c] += v;
        qy[c] += v * v;
        cy[c] += 1.0;
      }
  }
#pragma unroll
  for (int k = 0; k < kNin; ++k) {
    atomicAdd(&acc[k], s[k]);
    atomicAdd(&acc[kNin + k], q[k]);
  }
#pragma unroll
  for (int c = 0; c < kNout; ++c) {
    atomicAdd(&acc[2 * kNin + c], sy[c]);
    atomicAdd(&acc[2 * kNin + kNout + c], qy[c]);
    atomicAdd(&acc[2 * kNin + 2 * kNout + c], cy[c]);
  }
}

// order-preserving float <-> int mapping for atomic min/max
__device__ __forceinline__ int f2ord(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_mlp_box(const float *X, long long n, int *lo, int *hi) {
  int l[kNin], h[kNin];
#pragma unroll
  for (int k = 0; k < kNin; ++k) {
    l[k] = 0x7fffffff;
    h[k] = -0x7fffffff;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int k = 0; k < kNin; ++k) {
      const int v = f2ord(X[i * kNin + k]);
      l[k] = min(l[k], v);
      h[k] = max(h[k], v);
    }
#pragma unroll
  for (int k = 0; k < kNin; ++k) {
    atomicMin(&lo[k], l[k]);
    atomicMax(&hi[k], h[k]);
  }
}

// ------------------------------------------------------ features and targets
// The 12 features of a post-activation point (natural logarithms).
__device__ __forceinline__ void mlp_features(const ConstK<float> &K, const W<float> &w, float na, float wv,
                                             float f[kNin]) {
  const float ln2 = 0.693147180559945309f;
  f[0] = lg2a(fmaxf(w.qc, K.qmin)) * ln2;
  f[1] = lg2a(fmaxf(w.qr, K.qmin)) * ln2;
  f[2] = lg2a(fmaxf(w.nc, 1.f)) * ln2;
  f[3] = lg2a(fmaxf(w.nr, 1e-3f)) * ln2;
  f[4] = lg2a(w.rho) * ln2;
  f[5] = w.tc;
  f[6] = lg2a(w.p) * ln2;
  f[7] = lg2a(fmaxf(w.qv, 1e-10f)) * ln2;
  f[8] = wv;
  f[9] = lg2a(fmaxf(na, 1.f)) * ln2;
  f[10] = w.qc > K.qmin ? 1.f : 0.f;
  f[11] = w.qr > K.qmin ? 1.f : 0.f;
}

struct FeatArgs {
  int mode;               // 0: training data (raw features, log-rates, masks); 1: inference rows
  long long cap;          // rows available
  unsigned long long *rows;   // row counter
  float *X, *Y, *M;       // mode 0: [cap][12], [cap][4], [cap][4]
  __nv_bfloat16 *xb;      // mode 1: [cap][16] standardised BF16 features
  long long *rowpt;       // point index (k * pitch + c) of each row (mode 0: optional)
  float4 *surr;           // mode 1: [nlev][pitch]; NaN written where the point is outside the box
  const float *norm;      // mode 1: means and deviations of the features
  const float *box;       // mode 1: [12 lo][12 hi]
};

// The features of one point (index pt of its domain's [nlev][pitch] grid;
// gpt: its index in the rates array, which is pt for one domain): adjustment
// and activation as the mixed step does them, then the point's features (and,
// for training data, the scheme's four log-rates).  warm: the point gets a row.
__device__ __forceinline__ void feature_point(const KArgs &a, const KParams &P, const FeatArgs &fa, long long pt,
                                              long long gpt, bool &warm, float f[kNin], float y[kNout],
                                              float mk[kNout]) {
  const long long np = (long long)a.nlev * a.pitch;
  if (pt < np) {
    const int c = (int)(pt % a.pitch);
    if (c < a.ncols) {
      const ConstK<float> &K = P.f;
      Pt s;
      const double *b = a.fld + pt;
      const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
      s.T = b[0]; s.qv = b[1 * fs]; s.qc = b[2 * fs]; s.qr = b[3 * fs];
      s.qi = b[4 * fs]; s.qs = b[5 * fs]; s.qg = b[6 * fs];
      s.p = b[13 * fs];
      W<float> w;
      float es0, qs0;
      if (Mix::active(K, s, P.T0, w, es0, qs0)) {
        s.nc = b[7 * fs]; s.nr = b[8 * fs]; s.ni = b[9 * fs]; s.ns = b[10 * fs]; s.ng = b[11 * fs];
        s.na = b[12 * fs]; s.rho = b[14 * fs]; s.w = b[15 * fs];
        MixInc o;
        const float dn = Mix::pre(K, s, w, es0, qs0, o);
        warm = w.qc > K.qmin || w.qr > K.qmin;
        if (warm) {
          mlp_features(K, w, d2f(s.na) - dn, d2f(s.w), f);
          if (fa.mode == 0) {
            Rt<float> r;
            Phys<PolicyMix>::rates(K, w, a.dt, r);
            const bool hc = w.qc > K.qmin, hr = w.qr > K.qmin;
            const float v[kNout] = {r.aut, r.acc, r.scc, r.scr};
            const bool def[kNout] = {hc, hc && hr, hc, hr};
#pragma unroll
            for (int j = 0; j < kNout; ++j)
              if (def[j] && v[j] > 0.f) {
                y[j] = lg2a(v[j]) * 0.693147180559945309f;
                mk[j] = 1.f;
              }
          } else {
            bool inbox = true;
#pragma unroll
            for (int j = 0; j < kNin; ++j) inbox &= f[j] >= fa.box[j] && f[j] <= fa.box[kNin + j];
            if (!inbox) {
              fa.surr[gpt] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
              warm = false;
            }
          }
        }
      }
    }
  }
}

// Block-aggregated append of the rows: one atomic on the row counter per
// block (a counter that every warp hits serialises in L2), the warps' offsets
// from a prefix sum of their counts; rows come in no set order (each carries
// its point, gpt).  Every thread of the block calls it.
__device__ __forceinline__ void feature_append(const FeatArgs &fa, bool warm, long long gpt, const float f[kNin],
                                               const float y[kNout], const float mk[kNout]) {
  __shared__ unsigned s_off[256 / 32];
  __shared__ unsigned long long s_base;
  const unsigned ball = __ballot_sync(0xffffffffu, warm);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_off[wid] = __popc(ball);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      const unsigned t = s_off[i];
      s_off[i] = tot;
      tot += t;
    }
    s_base = tot ? atomicAdd(fa.rows, (unsigned long long)tot) : 0ull;
  }
  __syncthreads();
  if (!warm) return;
  const long long row = (long long)(s_base + s_off[wid]) + __popc(ball & ((1u << lane) - 1u));
  if (row >= fa.cap) return;   // the caller sees rows > cap and reports it
  if (fa.mode == 0) {
    if (fa.rowpt) fa.rowpt[row] = gpt;
#pragma unroll
    for (int j = 0; j < kNin; ++j) fa.X[row * kNin + j] = f[j];
#pragma unroll
    for (int j = 0; j < kNout; ++j) {
      fa.Y[row * kNout + j] = y[j];
      fa.M[row * kNout + j] = mk[j];
    }
  } else {
    __align__(16) __nv_bfloat16 hb[kNinPad];
#pragma unroll
    for (int j = 0; j < kNinPad; ++j)
      hb[j] = __float2bfloat16(j < kNin ? (f[j] - fa.norm[j]) / fa.norm[kNin + j] : 0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(fa.xb + row * kNinPad);
    dst[0] = reinterpret_cast<const uint4 *>(hb)[0];
    dst[1] = reinterpret_cast<const uint4 *>(hb)[1];
    fa.rowpt[row] = gpt;
  }
}

// One thread per point of a domain.
__global__ void __launch_bounds__(256) k_mlp_features(const KArgs a, const KParams P, const FeatArgs fa) {
  const long long pt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool warm = false;
  float f[kNin];
  float y[kNout] = {0, 0, 0, 0}, mk[kNout] = {0, 0, 0, 0};
  feature_point(a, P, fa, pt, pt, warm, f, y, mk);
  feature_append(fa, warm, pt, f, y, mk);
}

// One thread per point of every domain of a batch: the points of domain d
// are [dom[d].pt_off, dom[d].pt_off + nlev pitch) of the batch's rates array
// (a binary search over the domains' offsets finds a thread's domain).
__global__ void __launch_bounds__(256) k_mlp_features_batch(const DomDesc *dom, int ndom, long long total,
                                                            double dt, const KParams P, const FeatArgs fa) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool warm = false;
  float f[kNin];
  float y[kNout] = {0, 0, 0, 0}, mk[kNout] = {0, 0, 0, 0};
  if (g < total) {
    int lo = 0, hi = ndom - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (dom[mid].pt_off <= g) lo = mid;
      else hi = mid - 1;
    }
    const DomDesc d = dom[lo];
    KArgs a;
    a.fld = d.fld;
    a.pitch = d.pitch;
    a.dz = d.dz;
    a.precip = d.precip;
    a.err = nullptr;
    a.ncols = d.ncols;
    a.nlev = d.nlev;
    a.dt = dt;
    a.surr = nullptr;
    a.stats = nullptr;
    feature_point(a, P, fa, g - d.pt_off, g, warm, f, y, mk);
  }
  feature_append(fa, warm, g, f, y, mk);
}

// network outputs (standardised log-rates) -> rates at the rows' points
__global__ void k_mlp_scatter(const float *Yn, long long rows, const long long *rowpt, const float *norm,
                              float4 *surr, long long npts, unsigned *err) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  if (!CASIM_INDEX_OK(rowpt[r] >= 0 && rowpt[r] < npts, err)) return;
  const float *muy = norm + 2 * kNin, *sdy = norm + 2 * kNin + kNout;
  float v[kNout];
#pragma unroll
  for (int j = 0; j < kNout; ++j) v[j] = __expf(Yn[r * kNout + j] * sdy[j] + muy[j]);
  surr[rowpt[r]] = make_float4(v[0], v[1], v[2], v[3]);
}

}  // namespace casim_dev

// ------------------------------------------------ tcgen05 inference kernel
#include "casim_umma.cuh"

namespace casim_dev {

// Weight images in global memory, already in the swizzled shared-memory
// layout, so that 1-D bulk copies land them ready for the tensor cores:
//   W1: [256 rows][64] (k >= 12 zero)                                32 KB
//   W2, W3: four chunks each, chunk s = all 256 output rows x k = 64s..64s+63
//           (one K-slab)                                              32 KB each
//   W4: [16 rows][256] (rows >= 4 zero)                               8 KB
constexpr uint32_t kImgW1 = 256 * 128, kImgChunk = 256 * 128, kImgW4 = 16 * 4 * 128;
constexpr int kImgChunks = 8;
constexpr uint32_t kImgBytes = kImgW1 + kImgChunks * kImgChunk + kImgW4;

__global__ void k_mlp_images(const float *theta, unsigned char *img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  if (i < 256 * 64) {   // W1 (n, k)
    const int n = i / 64, k = i % 64;
    *reinterpret_cast<__nv_bfloat16 *>(img + sw128_offset(256, n, k)) =
        k < kNin ? __float2bfloat16(theta[kOffW1 + k * kNh + n]) : z;
  }
  if (i < 256 * 256) {  // W2, W3 (n, k)
    const int n = i / 256, k = i % 256, s = k >> 6;
    const uint32_t off = (uint32_t)s * kImgChunk + sw128_offset(256, n, k & 63);
    *reinterpret_cast<__nv_bfloat16 *>(img + kImgW1 + off) = __float2bfloat16(theta[kOffW2 + k * kNh + n]);
    *reinterpret_cast<__nv_bfloat16 *>(img + kImgW1 + 4 * kImgChunk + off) = __float2bfloat16(theta[kOffW3 + k * kNh + n]);
  }
  if (i < 16 * 256) {   // W4 (n, k)
    const int n = i / 256, k = i % 256;
    *reinterpret_cast<__nv_bfloat16 *>(img + kImgW1 + kImgChunks * kImgChunk + sw128_offset(16, n, k)) =
        n < kNout ? __float2bfloat16(theta[kOffW4 + k * kNout + n]) : z;
  }
}

struct UmmaArgs {
  const __nv_bfloat16 *xb;     // [rows][16] standardised features
  long long rows;              // rows, or the capacity when rows_dev is set
  const unsigned long long *rows_dev;   // if set: the row count, read on the device (at most rows)
  const long long *rowpt;      // point of each row (null: write Y rows instead)
  const unsigned char *img;    // weight images
  const float *theta;          // biases are read from the flat parameters
  const float *norm;           // output standardisation
  float4 *surr;                // rates at the points
  long long npts;              // points of surr (the rows' point indices are below it)
  float *y;                    // [rows][4] standardised outputs when rowpt is null
  unsigned *err;
};

constexpr unsigned kUmmaSpins = 1u << 22;
constexpr int kUmmaEpiWarps = 16;                       // 4 per TMEM lane quarter
constexpr int kUmmaMmaWarp = kUmmaEpiWarps;             // issues the MMAs, owns TMEM
constexpr int kUmmaProdWarp = kUmmaEpiWarps + 1;        // streams the weight chunks
constexpr int kUmmaThreads = (kUmmaEpiWarps + 2) * 32;
constexpr int kUmmaStages = 4;                          // weight-chunk ring
// dynamic shared memory (1024-byte aligned): resident W1 and W4, the chunk
// ring.  Activations live in tensor memory.
constexpr uint32_t kSmW1 = 0, kSmW4 = kSmW1 + kImgW1, kSmRing = kSmW4 + kImgW4;
// tensor-memory columns: accumulators A0 (layers 1, 3) and A1 (layers 2, 4),
// each later overwritten in place by its layer's BF16 activations; the next
// tile's features sit in A1's last 8 columns
constexpr uint32_t kTmA0 = 0, kTmA1 = 256, kTmFeat = 504;
constexpr int kUmmaSmem = 1024 + kSmRing + kUmmaStages * kImgChunk;
static_assert(kUmmaSmem + 4096 <= 232448, "shared memory of the tensor-core kernel");

// Persistent, one CTA (18 warps) per SM, 128-row tiles.
//
// Tensor memory holds two 256-column FP32 accumulators used by alternate
// layers (layer 1 -> A0, 2 -> A1, 3 -> A0, 4 -> A1), so the MMAs of layer
// l+1 run while the epilogue of layer l still reads layer l's sums.  The
// activations never touch shared memory: each epilogue warp writes the BF16
// activations of the 16 sums it has just read back into the first 8 of
// those 16 columns (two per 32-bit column, even k in the low half), and the
// next layer's MMAs read their A operand from there (K-step kk of 16 at
// column 16 kk).  Shared memory only holds weights, and its bandwidth --
// which bounds these MMAs -- goes to the B operand:
//  * epilogue warps (16): warp w reads TMEM lanes 32(w%4).. (its rows) and
//    columns 16(w/4)..+15 of each 64-column slab; per slab s: bias, tanh,
//    BF16 pack, tcgen05.st in place, then one arrival on act[s];
//  * MMA warp (one thread): per slab s it waits act[s] and issues that
//    K-slab's MMAs of the next layer (N = 256, weights from the ring);
//    after the last slab it commits the accumulator to acc;
//  * producer warp (one thread): streams the 8 weight chunks of layers 2-3
//    per tile through the ring (full/free barriers).
// Weight traffic from L2 is 256 KB per tile.  N = 256 MMAs read each A slab once
// (N = 128 halves would read it twice): shared-memory operand bandwidth, not
// the tensor pipe, bounds these MMAs.
// Every wait is bounded and gives up once any thread of the CTA has set the
// abort flag; before the tensor memory is released and the CTA leaves, all
// MMAs, copies and arrivals from or to this CTA have completed.
__global__ void __launch_bounds__(kUmmaThreads, 1) k_mlp_umma(const UmmaArgs u) {
  extern __shared__ __align__(16) unsigned char sraw[];
  unsigned char *sm = sraw + ((1024 - (smem_addr(sraw) & 1023)) & 1023);
  __shared__ float s_bias[3 * kNh + kNout];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_bar[24];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long nrows = u.rows_dev ? min((long long)*u.rows_dev, u.rows) : u.rows;
  const long long ntiles = (nrows + 127) / 128;
  const long long cta = blockIdx.x, ncta = gridDim.x;
  const long long my_tiles = cta < ntiles ? (ntiles - 1 - cta) / ncta + 1 : 0;
  const uint32_t sb = smem_addr(sm);
  volatile int *abort = &s_abort;
  enum { B_W = 0, B_FEAT = 1, B_ACC = 2, B_ACT = 3, B_FULL = 7, B_FREE = 7 + kUmmaStages, B_DRAIN = 7 + 2 * kUmmaStages };
  const uint32_t bar0 = smem_addr(&s_bar[0]);
  auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  auto fail = [&]() {
    *abort = 1;
    atomicOr(u.err, 4u);
  };

  for (int i = tid; i < kNh; i += kUmmaThreads) {
    s_bias[i] = u.theta[kOffB1 + i];
    s_bias[kNh + i] = u.theta[kOffB2 + i];
    s_bias[2 * kNh + i] = u.theta[kOffB3 + i];
  }
  if (tid < kNout) s_bias[3 * kNh + tid] = u.theta[kOffB4 + tid];
  if (warp == kUmmaMmaWarp) {
    tmem_alloc(smem_addr(&s_tmem), 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    bar_init(bar(B_W), 1);
    bar_init(bar(B_FEAT), kUmmaEpiWarps);
    bar_init(bar(B_ACC), 1);
    for (int s = 0; s < 4; ++s) bar_init(bar(B_ACT + s), kUmmaEpiWarps);
    for (int s = 0; s < kUmmaStages; ++s) {
      bar_init(bar(B_FULL + s), 1);
      bar_init(bar(B_FREE + s), 1);
    }
    bar_init(bar(B_DRAIN), 1);
    bar_fence_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_tmem;

  if (warp == kUmmaProdWarp) {
    if (lane == 0) {
      bar_expect_tx(bar(B_W), kImgW1 + kImgW4);
      bulk_load(sb + kSmW1, u.img, kImgW1, bar(B_W));
      bulk_load(sb + kSmW4, u.img + kImgW1 + kImgChunks * kImgChunk, kImgW4, bar(B_W));
      // load i goes to stage i % S as that stage's (i / S)-th fill; from the
      // second fill on it waits until the MMAs of the previous fill have
      // completed
      const long long nch = my_tiles * kImgChunks;
      long long i = 0;
      for (; i < nch; ++i) {
        const int st = (int)(i % kUmmaStages);
        const long long fill = i / kUmmaStages;
        if (fill > 0 && !bar_wait_or_abort(bar(B_FREE + st), (uint32_t)((fill - 1) & 1), kUmmaSpins, abort)) {
          fail();
          break;
        }
        bar_expect_tx(bar(B_FULL + st), kImgChunk);
        const uint32_t dst = sb + kSmRing + (uint32_t)st * kImgChunk;
        const unsigned char *src = u.img + kImgW1 + (uint32_t)(i % kImgChunks) * kImgChunk;
        bulk_load(dst, src, kImgChunk, bar(B_FULL + st));
      }
      // drain: the copies into this CTA have landed (last fill of each
      // stage), and so have the commits of those fills
      bar_wait(bar(B_W), 0, kUmmaSpins);
      for (int st = 0; st < kUmmaStages && st < i; ++st) {
        const long long fills = (i - st + kUmmaStages - 1) / kUmmaStages;
        bar_wait(bar(B_FULL + st), (uint32_t)((fills - 1) & 1), kUmmaSpins);
        bar_wait_or_abort(bar(B_FREE + st), (uint32_t)((fills - 1) & 1), kUmmaSpins, abort);
      }
    }
    __syncwarp();
  } else if (warp == kUmmaMmaWarp) {
    if (lane == 0) {
      const uint32_t id256 = umma_idesc_bf16(128, 256), id16 = umma_idesc_bf16(128, 16);
      bool ok = bar_wait_or_abort(bar(B_W), 0, kUmmaSpins, abort);
      int nfeat = 0, nact = 0;
      long long chunk = 0;
      for (long long it = 0; ok && it < my_tiles; ++it) {
        ok = bar_wait_or_abort(bar(B_FEAT), (uint32_t)(nfeat++ & 1), kUmmaSpins, abort);
        if (!ok) break;
        tc_fence_after();
        // layer 1: features (tensor memory, k < 16) x W1 -> A0
        umma_bf16_ts(taddr + kTmA0, taddr + kTmFeat, umma_desc_sw128(sb + kSmW1), id256, 0u);
        umma_commit(bar(B_ACC));
        // layers 2 (A0 -> A1) and 3 (A1 -> A0), K-slab by K-slab
        for (int l = 0; ok && l < 2; ++l, ++nact) {
          const uint32_t dacc = taddr + (l == 0 ? kTmA1 : kTmA0), ain = taddr + (l == 0 ? kTmA0 : kTmA1);
          for (int s = 0; ok && s < 4; ++s) {
            ok = bar_wait_or_abort(bar(B_ACT + s), (uint32_t)(nact & 1), kUmmaSpins, abort);
            if (!ok) break;
            tc_fence_after();
            const int st = (int)(chunk % kUmmaStages);
            ok = bar_wait_or_abort(bar(B_FULL + st), (uint32_t)((chunk / kUmmaStages) & 1), kUmmaSpins, abort);
            if (!ok) break;
            tc_fence_after();
            const uint32_t wst = sb + kSmRing + (uint32_t)st * kImgChunk;
#pragma unroll
            for (int sub = 0; sub < 4; ++sub)
              umma_bf16_ts(dacc, ain + 64u * (uint32_t)s + 16u * (uint32_t)sub, umma_desc_sw128(wst + 32u * (uint32_t)sub),
                           id256, (s | sub) ? 1u : 0u);
            umma_commit(bar(B_FREE + st));
            ++chunk;
          }
          if (ok) umma_commit(bar(B_ACC));
        }
        // layer 4: A0 x W4 -> A1 columns 0..15
        for (int s = 0; ok && s < 4; ++s) {
          ok = bar_wait_or_abort(bar(B_ACT + s), (uint32_t)(nact & 1), kUmmaSpins, abort);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int sub = 0; sub < 4; ++sub)
            umma_bf16_ts(taddr + kTmA1, taddr + kTmA0 + 64u * (uint32_t)s + 16u * (uint32_t)sub,
                         umma_desc_sw128(sb + kSmW4 + 2048u * (uint32_t)s + 32u * (uint32_t)sub), id16,
                         (s | sub) ? 1u : 0u);
        }
        ++nact;
        if (ok) umma_commit(bar(B_ACC));
      }
      if (!ok) fail();
      // drain: every MMA this thread issued has completed
      umma_commit(bar(B_DRAIN));
      bar_wait(bar(B_DRAIN), 0, kUmmaSpins);
    }
    __syncwarp();
  } else {
    // epilogue warps
    const int q = warp & 3, j = warp >> 2;
    const int row = 32 * q + lane;
    const uint32_t tl = taddr + ((uint32_t)(32 * q) << 16);
    int nacc = 0;
    bool ok = true;
    uint4 f0 = make_uint4(0, 0, 0, 0), f1 = f0;
    auto load_features = [&](long long g) {
      f0 = make_uint4(0, 0, 0, 0);
      f1 = f0;
      const long long r = g * 128 + row;
      if (g < ntiles && r < nrows) {
        const uint4 *src = reinterpret_cast<const uint4 *>(u.xb + r * kNinPad);
        f0 = src[0];
        f1 = src[1];
      }
    };
    if (j == 0) load_features(cta);
    for (long long g = cta; ok && g < ntiles; g += ncta) {
      const long long r0 = g * 128;
      // every epilogue warp arrives: the next tile's layer-1 MMA (which
      // overwrites A0) waits until all of them have seen the previous
      // tile's last accumulator phase; the features go to tensor memory
      // (A1's last columns: the previous tile's layer-3 MMAs, which read
      // A1, have completed)
      if (j == 0) {
        const uint32_t fv[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
        tmem_st8(tl + kTmFeat, fv);
        tc_fence_before();
      }
      __syncwarp();
      if (lane == 0) bar_arrive(bar(B_FEAT));
      if (j == 0) load_features(g + ncta);
      for (int l = 0; l < 3; ++l) {
        ok = bar_wait_or_abort(bar(B_ACC), (uint32_t)(nacc++ & 1), kUmmaSpins, abort);
        if (!ok) break;
        tc_fence_after();
        const uint32_t tacc = tl + (l == 1 ? kTmA1 : kTmA0);
        const float *b = s_bias + l * kNh;
#pragma unroll 1
        for (int s = 0; s < 4; ++s) {
          const int c0 = 64 * s + 16 * j;
          float v[16];
          tmem_ld16(tacc + (uint32_t)c0, v);
          uint32_t hb[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 p = __floats2bfloat162_rn(tanh_approx(v[2 * i] + b[c0 + 2 * i]),
                                                          tanh_approx(v[2 * i + 1] + b[c0 + 2 * i + 1]));
            hb[i] = *reinterpret_cast<const uint32_t *>(&p);
          }
          tmem_st8(tacc + (uint32_t)c0, hb);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) bar_arrive(bar(B_ACT + s));
        }
      }
      if (!ok) break;
      ok = bar_wait_or_abort(bar(B_ACC), (uint32_t)(nacc++ & 1), kUmmaSpins, abort);
      if (!ok) break;
      tc_fence_after();
      if (j == 0) {
        float v[16];
        tmem_ld16(tl + kTmA1, v);
        tc_fence_before();
        if (r0 + row < nrows) {
          float y[kNout];
#pragma unroll
          for (int i = 0; i < kNout; ++i) y[i] = v[i] + s_bias[3 * kNh + i];
          if (u.rowpt && CASIM_INDEX_OK(u.rowpt[r0 + row] >= 0 && u.rowpt[r0 + row] < u.npts, u.err)) {
            const float *muy = u.norm + 2 * kNin, *sdy = u.norm + 2 * kNin + kNout;
            u.surr[u.rowpt[r0 + row]] = make_float4(__expf(y[0] * sdy[0] + muy[0]), __expf(y[1] * sdy[1] + muy[1]),
                                                    __expf(y[2] * sdy[2] + muy[2]), __expf(y[3] * sdy[3] + muy[3]));
          } else {
#pragma unroll
            for (int i = 0; i < kNout; ++i) u.y[(r0 + row) * kNout + i] = y[i];
          }
        }
      }
    }
    if (!ok) fail();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kUmmaMmaWarp) tmem_dealloc(taddr, 512);
}


// ------------------------------------------------ tcgen05 training GEMM
// The training GEMMs of the network on the fifth-generation tensor cores:
// C[m][n] = sum_k A(m, k) B(n, k), operands BF16 with the strides of
// GemmArgs, FP32 accumulators in tensor memory, the same fused epilogues as
// k_gemm.  Each operand is K-major (unit stride along k: the forward pass and
// the data gradients) or MN-major (unit stride along m or n: the weight
// gradients, whose k runs over the batch); both are staged in shared memory
// as the K-major 128-byte-swizzled slabs the MMA reads (sw128_offset), an
// MN-major tile being transposed in registers on the way (8 x 8 blocks).
//
// One CTA of 4 warps per 128 x 128 output tile (split K over blockIdx.z as
// for k_gemm); K advances in slabs of 64 through two shared-memory buffers:
// all threads load slab s + 1 into registers while the MMAs of slab s run,
// then wait (bounded) for the MMAs that last read the buffer before storing
// into it.  One thread issues the MMAs (M = 128, N = the tile's columns
// rounded up to 16, K = 16 each) and commits each slab to its buffer's
// mbarrier.  Epilogue: warp w reads tensor-memory lanes 32w.. (its rows),
// 32 columns at a time, and passes the 32 x 32 block through shared memory
// (the operand buffers, free once the last MMA completed) so that the
// epilogue's loads and stores run along n, coalesced.  A wait that gives up
// sets error bit 4, waits again for the MMAs it issued and releases the
// tensor memory.
constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 64;
constexpr uint32_t kTcTile = kTcBM * kTcBK * 2;              // one operand slab: 16 KB
constexpr int kTcSmem = 1024 + 4 * (int)kTcTile;              // A and B, two buffers, 1024-byte alignment
constexpr unsigned kTcSpins = 1u << 24;

// One thread's share of an operand slab: rows r0..r0+127 of the operand
// (row index m or n), k in [k0, k0 + 64) of [.., ke), zeros outside it.
// K-major (unit stride along k): 8 chunks of 8 k, consecutive threads along a
// row.  MN-major (unit stride along the rows): one 8 (rows) x 8 (k) block,
// as 8 chunks of 8 rows at one k, transposed into 8 chunks of 8 k at one row
// when stored.  tc_fetch issues the global loads, tc_put writes the slab in
// the swizzled K-major layout, so both operands' loads are in flight
// together.
struct TcFrag {
  uint4 v[8];
};

__device__ __forceinline__ void tc_fetch(TcFrag &fr, const __nv_bfloat16 *P, long long srow, long long sk, int nrows,
                                         int r0, int k0, int ke, int tid) {
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  if (sk == 1) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = tid + 128 * j, r = i >> 3, ch = i & 7;
      const int row = r0 + r, k = k0 + 8 * ch;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (row < nrows && k < ke) {
        const __nv_bfloat16 *src = P + (long long)row * srow + k;
        if (k + 8 <= ke) {
          v = __ldg(reinterpret_cast<const uint4 *>(src));
        } else {
          __align__(16) __nv_bfloat16 e[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) e[t] = k + t < ke ? src[t] : zero;
          v = *reinterpret_cast<const uint4 *>(e);
        }
      }
      fr.v[j] = v;
    }
  } else {
    const int rg = tid & 15, kg = tid >> 4;
    const int row = r0 + 8 * rg;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = k0 + 8 * kg + kk;
      uint4 u = make_uint4(0, 0, 0, 0);
      if (k < ke && row < nrows) {
        const __nv_bfloat16 *src = P + (long long)k * sk + row;
        if (row + 8 <= nrows) {
          u = __ldg(reinterpret_cast<const uint4 *>(src));
        } else {
          __align__(16) __nv_bfloat16 e[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) e[t] = row + t < nrows ? src[t] : zero;
          u = *reinterpret_cast<const uint4 *>(e);
        }
      }
      fr.v[kk] = u;
    }
  }
}

__device__ __forceinline__ void tc_put(unsigned char *dst, const TcFrag &fr, long long sk, int tid) {
  if (sk == 1) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = tid + 128 * j, r = i >> 3, ch = i & 7;
      *reinterpret_cast<uint4 *>(dst + sw128_offset(kTcBM, r, 8 * ch)) = fr.v[j];
    }
  } else {
    const int rg = tid & 15, kg = tid >> 4;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(fr.v);   // w[4 kk + j]: rows 2j, 2j + 1 at k kk
#pragma unroll
    for (int mm = 0; mm < 8; ++mm) {
      const unsigned sel = (mm & 1) ? 0x7632u : 0x5410u;   // high or low halves of the two words
      const int j = mm >> 1;
      uint4 o;
      o.x = __byte_perm(w[0 * 4 + j], w[1 * 4 + j], sel);
      o.y = __byte_perm(w[2 * 4 + j], w[3 * 4 + j], sel);
      o.z = __byte_perm(w[4 * 4 + j], w[5 * 4 + j], sel);
      o.w = __byte_perm(w[6 * 4 + j], w[7 * 4 + j], sel);
      *reinterpret_cast<uint4 *>(dst + sw128_offset(kTcBM, 8 * rg + mm, 8 * kg)) = o;
    }
  }
}

template <class Epi>
__global__ void __launch_bounds__(128) k_gemm_tc(const GemmArgs g, const Epi epi, unsigned *err) {
  extern __shared__ __align__(16) unsigned char sraw[];
  unsigned char *sm = sraw + ((1024 - (smem_addr(sraw) & 1023)) & 1023);
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_bar[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  const int kb = blockIdx.z * g.kchunk, ke = min(g.K, kb + g.kchunk);
  const int nst = ke > kb ? (ke - kb + kTcBK - 1) / kTcBK : 0;
  const int ncols = min(kTcBN, ((g.N - n0) + 15) / 16 * 16);   // MMA N: the tile's columns, multiple of 16
  const uint32_t idesc = umma_idesc_bf16(kTcBM, ncols);
  unsigned char *bufA[2] = {sm, sm + 2 * kTcTile};
  unsigned char *bufB[2] = {sm + kTcTile, sm + 3 * kTcTile};
  const uint32_t bar0 = smem_addr(&s_bar[0]);
  if (warp == 0) {
    tmem_alloc(smem_addr(&s_tmem), kTcBN);
    tmem_relinquish();
  }
  if (tid == 0) {
    bar_init(bar0, 1);
    bar_init(bar0 + 8, 1);
    bar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_tmem;
  bool ok = true;
  TcFrag fa, fb;
  if (nst > 0) {
    tc_fetch(fa, g.A, g.sam, g.sak, g.M, m0, kb, ke, tid);
    tc_fetch(fb, g.B, g.sbn, g.sbk, g.N, n0, kb, ke, tid);
    tc_put(bufA[0], fa, g.sak, tid);
    tc_put(bufB[0], fb, g.sbk, tid);
  }
  fence_async_smem();
  __syncthreads();
  for (int s = 0; s < nst; ++s) {
    const int buf = s & 1, k0 = kb + s * kTcBK;
    if (tid == 0) {
      tc_fence_after();
      const int nsub = (min(kTcBK, ke - k0) + 15) / 16;
      const uint32_t a = smem_addr(bufA[buf]), b = smem_addr(bufB[buf]);
      for (int sub = 0; sub < nsub; ++sub)
        umma_bf16(taddr, umma_desc_sw128(a + 32u * (uint32_t)sub), umma_desc_sw128(b + 32u * (uint32_t)sub), idesc,
                  (s | sub) ? 1u : 0u);
      umma_commit(bar0 + 8u * (uint32_t)buf);
    }
    if (s + 1 < nst) {
      const int nb = buf ^ 1;
      tc_fetch(fa, g.A, g.sam, g.sak, g.M, m0, k0 + kTcBK, ke, tid);
      tc_fetch(fb, g.B, g.sbn, g.sbk, g.N, n0, k0 + kTcBK, ke, tid);
      // the MMAs of slab s - 1 read buffer nb: wait for their commit
      if (s >= 1 && ok) ok = bar_wait(bar0 + 8u * (uint32_t)nb, (uint32_t)(((s - 1) >> 1) & 1), kTcSpins);
      if (ok) {
        tc_put(bufA[nb], fa, g.sak, tid);
        tc_put(bufB[nb], fb, g.sbk, tid);
      }
      fence_async_smem();
    }
    __syncthreads();
  }
  // the last slab's commit completes after every MMA of the tile
  if (nst > 0) {
    const int last = nst - 1;
    if (!bar_wait(bar0 + 8u * (uint32_t)(last & 1), (uint32_t)((last >> 1) & 1), kTcSpins)) ok = false;
  }
  tc_fence_after();
  if (!__all_sync(0xffffffffu, ok)) ok = false;
  if (ok) {
    float *blk = reinterpret_cast<float *>(sm) + warp * (32 * 33);
    for (int c0 = 0; c0 < ncols; c0 += 32) {
      float v[32];
      if (nst > 0) {
        tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 32; ++i) blk[lane * 33 + i] = v[i];   // row lane, column i
      __syncwarp();
      const int n = n0 + c0 + lane;
      if (c0 + lane < ncols && n < g.N) {
        if constexpr (Epi::kLoad) {
          // 16 rows at a time: their reads first, then the epilogue
#pragma unroll
          for (int h = 0; h < 32; h += 16) {
            float ld[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) {
              const int m = m0 + 32 * warp + h + r;
              ld[r] = m < g.M ? epi.load(m, n) : 0.f;
            }
#pragma unroll
            for (int r = 0; r < 16; ++r) {
              const int m = m0 + 32 * warp + h + r;
              if (m < g.M) epi.apply(m, n, blk[(h + r) * 33 + lane], ld[r]);
            }
          }
        } else {
#pragma unroll 8
          for (int r = 0; r < 32; ++r) {
            const int m = m0 + 32 * warp + r;
            if (m < g.M) epi(m, n, blk[r * 33 + lane]);
          }
        }
      }
    }
  } else if (lane == 0) {
    atomicOr(err, 4u);
  }
  tc_fence_before();
  __syncthreads();
  if (!ok && tid == 0 && nst > 0) {
    // drain: every MMA this CTA issued has completed before its tensor
    // memory is released (bounded as every wait)
    const int last = nst - 1;
    bar_wait(bar0 + 8u * (uint32_t)(last & 1), (uint32_t)((last >> 1) & 1), kTcSpins);
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, kTcBN);
}

}  // namespace casim_dev
