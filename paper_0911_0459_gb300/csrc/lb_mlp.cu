// Learned surrogate for l(t): ensemble MLP trained and evaluated by hand-written
// kernels (include/lb_mlp.h).
//
// Contractions: C = A B on tensor cores, mma.sync m16n8k16 with BF16 operands
// and FP32 accumulation.  A 64x64 tile per CTA (4 warps of 32x32), K in steps
// of 16 staged through shared memory; operands are addressed through element
// strides, so the transposed products of the backward pass need no copies.
// The weight gradients contract over the batch (K up to max_batch rows) into
// small outputs: they split K over blockIdx.z and add the FP32 partials in a
// fixed order afterwards (split-K, deterministic).
// Epilogues fuse the bias and tanh (forward), the tanh derivative (backward)
// and the BF16 rounding of activations.  Ensemble members run in the z
// dimension of every launch.  One training iteration (forward, loss, backward,
// AdamW) is captured once as a CUDA graph and replayed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "lb_mlp.h"

namespace {

typedef __nv_bfloat16 bf16;

enum { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_TANH = 2, EPI_DTANH = 3 };

struct GemmArgs {
  int M, N, K;
  const bf16* A;
  long sam, sak, a_mem;
  const bf16* B;
  long sbk, sbn, b_mem;
  int epi;
  const float* bias;
  long bias_mem;
  float* Cf;
  long ldcf, cf_mem;
  bf16* Cb;
  long ldcb, cb_mem;
  const bf16* H;  // activation whose tanh derivative multiplies (EPI_DTANH)
  long ldh, h_mem;
  int ks;         // K splits: blockIdx.z = member * ks + split; split s takes K rows [s kc, (s + 1) kc)
  int kc;
  long cf_split;  // offset of split s's partial output from split 0's
};

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g) {
  constexpr int TM = 64, TN = 64, TK = 16;
  __shared__ bf16 As[TM][TK + 8];
  __shared__ bf16 Bs[TK][TN + 8];
  const int mem = blockIdx.z / g.ks, split = blockIdx.z - mem * g.ks;
  const int kb = split * g.kc, ke = min(g.K, kb + g.kc);
  const bf16* A = g.A + mem * g.a_mem;
  const bf16* B = g.B + mem * g.b_mem;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  const bf16 zero = __float2bfloat16(0.0f);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;

  for (int k0 = kb; k0 < ke; k0 += TK) {
    // stage the A (TM x TK) and B (TK x TN) tiles; consecutive threads walk the
    // unit-stride direction of each operand
    for (int e = tid; e < TM * TK; e += 128) {
      int r, c;
      if (g.sam == 1) {
        r = e % TM;
        c = e / TM;
      } else {
        r = e / TK;
        c = e % TK;
      }
      const int m = m0 + r, k = k0 + c;
      As[r][c] = (m < g.M && k < ke) ? A[m * g.sam + k * g.sak] : zero;
    }
    for (int e = tid; e < TK * TN; e += 128) {
      int r, c;
      if (g.sbk == 1) {
        r = e % TK;
        c = e / TK;
      } else {
        r = e / TN;
        c = e % TN;
      }
      const int k = k0 + r, n = n0 + c;
      Bs[r][c] = (k < ke && n < g.N) ? B[k * g.sbk + n * g.sbn] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r = wm + mi * 16;
      uint32_t a[4];
      a[0] = pack2(As[r + gq][2 * tq], As[r + gq][2 * tq + 1]);
      a[1] = pack2(As[r + gq + 8][2 * tq], As[r + gq + 8][2 * tq + 1]);
      a[2] = pack2(As[r + gq][2 * tq + 8], As[r + gq][2 * tq + 9]);
      a[3] = pack2(As[r + gq + 8][2 * tq + 8], As[r + gq + 8][2 * tq + 9]);
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn + ni * 8 + gq;
        uint32_t b[2];
        b[0] = pack2(Bs[2 * tq][c], Bs[2 * tq + 1][c]);
        b[1] = pack2(Bs[2 * tq + 8][c], Bs[2 * tq + 9][c]);
        mma_bf16(acc[mi][ni], a, b);
      }
    }
    __syncthreads();
  }

  const float* bias = g.bias ? g.bias + mem * g.bias_mem : nullptr;
  float* Cf = g.Cf ? g.Cf + mem * g.cf_mem + split * g.cf_split : nullptr;
  bf16* Cb = g.Cb ? g.Cb + mem * g.cb_mem : nullptr;
  const bf16* H = g.H ? g.H + mem * g.h_mem : nullptr;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + mi * 16 + gq + (q >> 1) * 8;
        const int n = n0 + wn + ni * 8 + 2 * tq + (q & 1);
        if (m >= g.M || n >= g.N) continue;
        float v = acc[mi][ni][q];
        if (g.epi == EPI_BIAS_F32 || g.epi == EPI_BIAS_TANH) v += bias[n];
        if (g.epi == EPI_BIAS_TANH) v = tanhf(v);
        if (g.epi == EPI_DTANH) {
          const float h = __bfloat162float(H[(long)m * g.ldh + n]);
          v *= 1.0f - h * h;
        }
        if (Cf) Cf[(long)m * g.ldcf + n] = v;
        if (Cb) Cb[(long)m * g.ldcb + n] = __float2bfloat16(v);
      }
}

// dY = 2 (Y - T) / (n n_out) in FP32 and BF16; per-member loss accumulated.
// out[m][n] (row stride ldo, member stride o_mem) = sum over s = 0 .. ks - 1, in that
// order, of the split-K partials part[member][s][m][n] (dense M x N).
__global__ void splitk_sum_kernel(const float* __restrict__ part, int ks, int M, int N, float* out, long ldo,
                                  long o_mem) {
  const int mem = blockIdx.y;
  const long MN = (long)M * N;
  const float* pm = part + (long)mem * ks * MN;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < MN; e += (long)gridDim.x * blockDim.x) {
    float v = 0.0f;
    for (int s = 0; s < ks; ++s) v += pm[s * MN + e];
    out[mem * o_mem + (e / N) * ldo + (e % N)] = v;
  }
}

__global__ void loss_grad_kernel(const float* Y, const float* T, int n, int nout, long mem_stride, float* dYf,
                                 bf16* dYb, float* loss) {
  const int mem = blockIdx.y;
  const float scale = 1.0f / ((float)n * (float)nout);
  float acc = 0.0f;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * nout; e += (long)gridDim.x * blockDim.x) {
    const float d = Y[mem * mem_stride + e] - T[e];
    acc += d * d;
    const float gr = 2.0f * d * scale;
    dYf[mem * mem_stride + e] = gr;
    dYb[mem * mem_stride + e] = __float2bfloat16(gr);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += sh[w];
    atomicAdd(&loss[mem], s * scale);
  }
}

// out[mem][c] = sum over rows of X[mem][r][c] (bias gradients).
__global__ void colsum_kernel(const float* X, int rows, int cols, long x_mem, float* out, long out_mem) {
  const int mem = blockIdx.y;
  const int c = blockIdx.x;
  float acc = 0.0f;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) acc += X[mem * x_mem + (long)r * cols + c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += sh[w];
    out[mem * out_mem + c] = s;
  }
}

struct Sched {
  int t;        // updates done
  int total;    // length of the cosine schedule
  float lr0, lr_min, wd;
};

// AdamW on every member: FP32 master weights, BF16 working copy.  weight_mask
// marks which parameter ranges are weights (decayed) and which are biases.
__global__ void adamw_kernel(float* p, bf16* pb, const float* gr, float* m1, float* m2, long P, const Sched* sc,
                             long b1, long w2, long b2, long w3, long b3) {
  const int mem = blockIdx.y;
  const int t = sc->t + 1;
  const float pi = 3.14159265358979f;
  const float frac = sc->total > 1 ? fminf((float)(t - 1) / (float)(sc->total - 1), 1.0f) : 1.0f;
  const float lr = sc->lr_min + 0.5f * (sc->lr0 - sc->lr_min) * (1.0f + cosf(pi * frac));
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
    const long j = mem * P + i;
    const float gv = gr[j];
    const float a = beta1 * m1[j] + (1.0f - beta1) * gv;
    const float b = beta2 * m2[j] + (1.0f - beta2) * gv * gv;
    m1[j] = a;
    m2[j] = b;
    const bool weight = (i < b1) || (i >= w2 && i < b2) || (i >= w3 && i < b3);
    float pv = p[j];
    if (weight) pv -= lr * sc->wd * pv;
    pv -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    p[j] = pv;
    pb[j] = __float2bfloat16(pv);
  }
}

__global__ void advance_kernel(Sched* sc) { sc->t += 1; }

// x (FP32, [n][n_in]) -> BF16 [n][16] with zero padding.
__global__ void pack_x_kernel(const float* x, int n, int nin, bf16* xb) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * 16; e += (long)gridDim.x * blockDim.x) {
    const long r = e / 16;
    const int c = (int)(e % 16);
    xb[e] = __float2bfloat16(c < nin ? x[r * nin + c] : 0.0f);
  }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Glorot-uniform weights (counter-based generator), zero biases.
__global__ void init_params_kernel(float* p, bf16* pb, long P, unsigned long long seed, int nin, int nh, int nout) {
  const int mem = blockIdx.y;
  const long b1 = (long)nh * nin, w2 = b1 + nh, b2 = w2 + (long)nh * nh, w3 = b2 + nh, b3 = w3 + (long)nout * nh;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
    float a = 0.0f;
    if (i < b1)
      a = sqrtf(6.0f / (nin + nh));
    else if (i >= w2 && i < b2)
      a = sqrtf(6.0f / (nh + nh));
    else if (i >= w3 && i < b3)
      a = sqrtf(6.0f / (nh + nout));
    const unsigned long long r = mix64((seed + mem) * 0x100000001B3ull + (unsigned long long)i);
    const float u = (float)((r >> 11) * (1.0 / 9007199254740992.0));  // [0, 1)
    const float v = a * (2.0f * u - 1.0f);
    p[mem * P + i] = v;
    pb[mem * P + i] = __float2bfloat16(v);
  }
}

// mean and standard deviation over members of Y [K][n][nout].
__global__ void ensemble_kernel(const float* Y, int K, long stride, long count, float* mean, float* sd) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < count; e += (long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int k = 0; k < K; ++k) s += Y[k * stride + e];
    const float mu = s / K;
    float q = 0.0f;
    for (int k = 0; k < K; ++k) {
      const float d = Y[k * stride + e] - mu;
      q += d * d;
    }
    mean[e] = mu;
    sd[e] = K > 1 ? sqrtf(q / (K - 1)) : 0.0f;
  }
}

thread_local char g_mlp_err[512] = "";

}  // namespace

struct lb_mlp {
  int nin, nh, nout, K, maxb;
  long P;
  long ow1, ob1, ow2, ob2, ow3, ob3;
  cudaStream_t stream, cap;
  lb_alloc alloc;
  int have_alloc;
  std::vector<void*> owned;
  float *p, *g, *m1, *m2;
  bf16* pb;
  Sched* sched;
  float* loss;
  // activations (per member)
  bf16 *xb, *xbp, *h1, *h2, *dyb, *dz2b, *dz1b;
  float *y, *dyf, *dz2f, *dz1f, *t;
  float* part;  // split-K partials of the weight gradients
  int ks_max;   // largest K split the partial buffer holds
  int n;  // rows of the loaded data
  cudaGraphExec_t gexec;
  int graph_n;
  char err[512];
};

static void merr(lb_mlp* m, const char* fmt, ...) {
  char* dst = m ? m->err : g_mlp_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
}

#define MCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      merr(m, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return LB_ERR_CUDA;                                                                  \
    }                                                                                      \
  } while (0)

static void* malloc_dev(lb_mlp* m, size_t bytes) {
  void* p = NULL;
  if (m->have_alloc)
    p = m->alloc.malloc_fn(bytes, (void*)m->stream, m->alloc.user);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = NULL;
  }
  if (p) m->owned.push_back(p);
  return p;
}

static cudaError_t gemm(lb_mlp* m, cudaStream_t s, int M, int N, int K, const bf16* A, long sam, long sak,
                        long a_mem, const bf16* B, long sbk, long sbn, long b_mem, int epi, const float* bias,
                        long bias_mem, float* Cf, long ldcf, long cf_mem, bf16* Cb, long ldcb, long cb_mem,
                        const bf16* H, long ldh, long h_mem) {
  GemmArgs g = {M, N, K, A, sam, sak, a_mem, B, sbk, sbn, b_mem, epi, bias, bias_mem,
                Cf, ldcf, cf_mem, Cb, ldcb, cb_mem, H, ldh, h_mem, 1, K, 0};
  dim3 grid((N + 63) / 64, (M + 63) / 64, m->K);
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
  return cudaGetLastError();
}

// A weight gradient C (M x N, FP32, row stride ldc, member stride c_mem) = A B with K
// the batch: split-K over about 128 rows per split when K is long, then the fixed-order
// sum of the partials into C.
static cudaError_t gemm_wgrad(lb_mlp* m, cudaStream_t s, int M, int N, int K, const bf16* A, long sam, long sak,
                              long a_mem, const bf16* B, long sbk, long sbn, long b_mem, float* C, long ldc,
                              long c_mem) {
  int ks = (K + 127) / 128;
  if (ks > m->ks_max) ks = m->ks_max;
  if (ks <= 1)
    return gemm(m, s, M, N, K, A, sam, sak, a_mem, B, sbk, sbn, b_mem, EPI_F32, NULL, 0, C, ldc, c_mem, NULL, 0, 0,
                NULL, 0, 0);
  const int kc = ((K + ks - 1) / ks + 15) / 16 * 16;
  ks = (K + kc - 1) / kc;
  const long MN = (long)M * N;
  GemmArgs g = {M, N, K, A, sam, sak, a_mem, B, sbk, sbn, b_mem, EPI_F32, NULL, 0,
                m->part, N, ks * MN, NULL, 0, 0, NULL, 0, 0, ks, kc, MN};
  dim3 grid((N + 63) / 64, (M + 63) / 64, m->K * ks);
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  const long blocks = (MN + 255) / 256;
  splitk_sum_kernel<<<dim3((unsigned)(blocks < 1024 ? blocks : 1024), m->K), 256, 0, s>>>(m->part, ks, M, N, C, ldc,
                                                                                          c_mem);
  return cudaGetLastError();
}

// forward of every member on rows [0, n) of the packed inputs xb; outputs in m->y
static cudaError_t forward(lb_mlp* m, int n, const bf16* xb, cudaStream_t s) {
  const long H = m->nh, O = m->nout, B = m->maxb;
  cudaError_t e;
  e = gemm(m, s, n, m->nh, m->nin, xb, 16, 1, 0, m->pb + m->ow1, 1, m->nin, m->P, EPI_BIAS_TANH, m->p + m->ob1, m->P,
           NULL, 0, 0, m->h1, H, B * H, NULL, 0, 0);
  if (e) return e;
  e = gemm(m, s, n, m->nh, m->nh, m->h1, H, 1, B * H, m->pb + m->ow2, 1, H, m->P, EPI_BIAS_TANH, m->p + m->ob2, m->P,
           NULL, 0, 0, m->h2, H, B * H, NULL, 0, 0);
  if (e) return e;
  return gemm(m, s, n, m->nout, m->nh, m->h2, H, 1, B * H, m->pb + m->ow3, 1, H, m->P, EPI_BIAS_F32, m->p + m->ob3,
              m->P, m->y, O, B * O, NULL, 0, 0, NULL, 0, 0);
}

// forward, loss and gradients of every member on the loaded data (grads in m->g)
static cudaError_t backward(lb_mlp* m, cudaStream_t s) {
  const int n = m->n;
  const long H = m->nh, O = m->nout, B = m->maxb;
  cudaError_t e = forward(m, n, m->xb, s);
  if (e) return e;
  e = cudaMemsetAsync(m->loss, 0, m->K * sizeof(float), s);
  if (e) return e;
  loss_grad_kernel<<<dim3(64, m->K), 256, 0, s>>>(m->y, m->t, n, m->nout, B * O, m->dyf, m->dyb, m->loss);
  if ((e = cudaGetLastError())) return e;
  // dW3 = dY^T H2, db3 = colsum dY
  e = gemm_wgrad(m, s, m->nout, m->nh, n, m->dyb, 1, O, B * O, m->h2, H, 1, B * H, m->g + m->ow3, H, m->P);
  if (e) return e;
  colsum_kernel<<<dim3(m->nout, m->K), 256, 0, s>>>(m->dyf, n, m->nout, B * O, m->g + m->ob3, m->P);
  if ((e = cudaGetLastError())) return e;
  // dZ2 = (dY W3) * (1 - H2^2)
  e = gemm(m, s, n, m->nh, m->nout, m->dyb, O, 1, B * O, m->pb + m->ow3, H, 1, m->P, EPI_DTANH, NULL, 0, m->dz2f, H,
           B * H, m->dz2b, H, B * H, m->h2, H, B * H);
  if (e) return e;
  // dW2 = dZ2^T H1, db2
  e = gemm_wgrad(m, s, m->nh, m->nh, n, m->dz2b, 1, H, B * H, m->h1, H, 1, B * H, m->g + m->ow2, H, m->P);
  if (e) return e;
  colsum_kernel<<<dim3(m->nh, m->K), 256, 0, s>>>(m->dz2f, n, m->nh, B * H, m->g + m->ob2, m->P);
  if ((e = cudaGetLastError())) return e;
  // dZ1 = (dZ2 W2) * (1 - H1^2)
  e = gemm(m, s, n, m->nh, m->nh, m->dz2b, H, 1, B * H, m->pb + m->ow2, H, 1, m->P, EPI_DTANH, NULL, 0, m->dz1f, H,
           B * H, m->dz1b, H, B * H, m->h1, H, B * H);
  if (e) return e;
  // dW1 = dZ1^T X, db1
  e = gemm_wgrad(m, s, m->nh, m->nin, n, m->dz1b, 1, H, B * H, m->xb, 16, 1, 0, m->g + m->ow1, m->nin, m->P);
  if (e) return e;
  colsum_kernel<<<dim3(m->nh, m->K), 256, 0, s>>>(m->dz1f, n, m->nh, B * H, m->g + m->ob1, m->P);
  return cudaGetLastError();
}

static cudaError_t train_step(lb_mlp* m, cudaStream_t s) {
  cudaError_t e = backward(m, s);
  if (e) return e;
  adamw_kernel<<<dim3(64, m->K), 256, 0, s>>>(m->p, m->pb, m->g, m->m1, m->m2, m->P, m->sched, m->ob1, m->ow2,
                                               m->ob2, m->ow3, m->ob3);
  if ((e = cudaGetLastError())) return e;
  advance_kernel<<<1, 1, 0, s>>>(m->sched);
  return cudaGetLastError();
}

extern "C" {

lb_status lb_mlp_create(int nin, int nh, int nout, int members, int max_batch, unsigned long long seed,
                        const lb_alloc* alloc, void* stream, lb_mlp** out) {
  lb_mlp* m = NULL;
  if (!out) return LB_ERR_ARG;
  *out = NULL;
  if (nin < 1 || nin > 16 || nh < 64 || nh % 64 || nh > 1024 || nout < 8 || nout % 8 || nout > 1024 || members < 1 ||
      members > 16 || max_batch < 1 || max_batch > 65535 * 64)  // row tiles of 64 on gridDim.y
    return merr(NULL, "invalid network shape"), LB_ERR_ARG;
  if (alloc && (!alloc->malloc_fn || !alloc->free_fn)) return merr(NULL, "incomplete allocator"), LB_ERR_ARG;
  m = new (std::nothrow) lb_mlp();
  if (!m) return LB_ERR_NOMEM;
  m->nin = nin; m->nh = nh; m->nout = nout; m->K = members; m->maxb = max_batch;
  m->ow1 = 0; m->ob1 = (long)nh * nin; m->ow2 = m->ob1 + nh; m->ob2 = m->ow2 + (long)nh * nh;
  m->ow3 = m->ob2 + nh; m->ob3 = m->ow3 + (long)nout * nh;
  m->P = m->ob3 + nout;
  m->stream = (cudaStream_t)stream;
  m->have_alloc = alloc != NULL;
  if (alloc) m->alloc = *alloc;
  if (cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete m;
    return merr(NULL, "cudaStreamCreate failed"), LB_ERR_CUDA;
  }
  const long PK = m->P * members, B = max_batch;
  m->p = (float*)malloc_dev(m, PK * 4);
  m->g = (float*)malloc_dev(m, PK * 4);
  m->m1 = (float*)malloc_dev(m, PK * 4);
  m->m2 = (float*)malloc_dev(m, PK * 4);
  m->pb = (bf16*)malloc_dev(m, PK * 2);
  m->sched = (Sched*)malloc_dev(m, sizeof(Sched));
  m->loss = (float*)malloc_dev(m, 64 * sizeof(float));
  m->xb = (bf16*)malloc_dev(m, B * 16 * 2);
  m->xbp = (bf16*)malloc_dev(m, B * 16 * 2);
  m->h1 = (bf16*)malloc_dev(m, members * B * nh * 2);
  m->h2 = (bf16*)malloc_dev(m, members * B * nh * 2);
  m->dz2b = (bf16*)malloc_dev(m, members * B * nh * 2);
  m->dz1b = (bf16*)malloc_dev(m, members * B * nh * 2);
  m->dz2f = (float*)malloc_dev(m, members * B * nh * 4);
  m->dz1f = (float*)malloc_dev(m, members * B * nh * 4);
  m->y = (float*)malloc_dev(m, members * B * nout * 4);
  m->dyf = (float*)malloc_dev(m, members * B * nout * 4);
  m->dyb = (bf16*)malloc_dev(m, members * B * nout * 2);
  m->t = (float*)malloc_dev(m, B * nout * 4);
  // split-K partials of the largest weight gradient (nh x max(nh, nout)), about 128
  // batch rows per split, at most 32 splits and 256 MB
  {
    const long mn = (long)nh * (nh > nout ? nh : nout);
    long ks = (B + 127) / 128;
    if (ks > 32) ks = 32;
    const long cap = (256L << 20) / (4L * members * mn);
    if (ks > cap) ks = cap;
    m->ks_max = ks > 1 ? (int)ks : 1;
    m->part = m->ks_max > 1 ? (float*)malloc_dev(m, 4L * members * m->ks_max * mn) : NULL;
  }
  bool ok = (m->ks_max == 1 || m->part) && m->p && m->g && m->m1 && m->m2 && m->pb && m->sched && m->loss && m->xb && m->xbp && m->h1 && m->h2 && m->dz2b &&
            m->dz1b && m->dz2f && m->dz1f && m->y && m->dyf && m->dyb && m->t;
  if (!ok) {
    lb_mlp_destroy(m);
    return merr(NULL, "device allocation failed"), LB_ERR_NOMEM;
  }
  init_params_kernel<<<dim3(64, members), 256, 0, m->stream>>>(m->p, m->pb, m->P, seed, nin, nh, nout);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m1, 0, PK * 4, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m2, 0, PK * 4, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->sched, 0, sizeof(Sched), m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    merr(NULL, "init failed: %s", cudaGetErrorString(e));
    lb_mlp_destroy(m);
    return LB_ERR_CUDA;
  }
  *out = m;
  return LB_OK;
}

void lb_mlp_destroy(lb_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  if (m->gexec) cudaGraphExecDestroy(m->gexec);
  for (void* p : m->owned) {
    if (m->have_alloc)
      m->alloc.free_fn(p, (void*)m->stream, m->alloc.user);
    else
      cudaFree(p);
  }
  if (m->cap) cudaStreamDestroy(m->cap);
  delete m;
}

long lb_mlp_num_params(const lb_mlp* m) { return m ? m->P : -1; }

lb_status lb_mlp_get_params(lb_mlp* m, int k, float* params) {
  if (!m || k < 0 || k >= m->K || !params) return LB_ERR_ARG;
  MCK(cudaMemcpyAsync(params, m->p + k * m->P, m->P * 4, cudaMemcpyDeviceToHost, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  return LB_OK;
}

lb_status lb_mlp_set_params(lb_mlp* m, int k, const float* params) {
  if (!m || k < 0 || k >= m->K || !params) return LB_ERR_ARG;
  std::vector<bf16> hb(m->P);
  for (long i = 0; i < m->P; ++i) hb[i] = __float2bfloat16(params[i]);
  MCK(cudaMemcpyAsync(m->p + k * m->P, params, m->P * 4, cudaMemcpyHostToDevice, m->stream));
  MCK(cudaMemcpyAsync(m->pb + k * m->P, hb.data(), m->P * 2, cudaMemcpyHostToDevice, m->stream));
  MCK(cudaMemsetAsync(m->m1 + k * m->P, 0, m->P * 4, m->stream));
  MCK(cudaMemsetAsync(m->m2 + k * m->P, 0, m->P * 4, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  return LB_OK;
}

lb_status lb_mlp_set_data(lb_mlp* m, int n, const float* x, const float* y) {
  if (!m || n < 1 || n > m->maxb || !x || !y) return LB_ERR_ARG;
  float* dx = (float*)malloc_dev(m, (size_t)n * m->nin * 4);
  if (!dx) return merr(m, "device allocation failed"), LB_ERR_NOMEM;
  MCK(cudaMemcpyAsync(dx, x, (size_t)n * m->nin * 4, cudaMemcpyHostToDevice, m->stream));
  pack_x_kernel<<<64, 256, 0, m->stream>>>(dx, n, m->nin, m->xb);
  MCK(cudaGetLastError());
  MCK(cudaMemcpyAsync(m->t, y, (size_t)n * m->nout * 4, cudaMemcpyHostToDevice, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  if (m->have_alloc)
    m->alloc.free_fn(dx, (void*)m->stream, m->alloc.user);
  else
    cudaFree(dx);
  m->owned.pop_back();
  m->n = n;
  if (m->gexec) {
    cudaGraphExecDestroy(m->gexec);
    m->gexec = NULL;
  }
  return LB_OK;
}

lb_status lb_mlp_gradients(lb_mlp* m, int k, float* grads, float* loss) {
  if (!m || k < 0 || k >= m->K || !grads || m->n < 1) return LB_ERR_ARG;
  MCK(backward(m, m->stream));
  MCK(cudaMemcpyAsync(grads, m->g + k * m->P, m->P * 4, cudaMemcpyDeviceToHost, m->stream));
  float hl[64];
  MCK(cudaMemcpyAsync(hl, m->loss, m->K * 4, cudaMemcpyDeviceToHost, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  if (loss) *loss = hl[k];
  return LB_OK;
}

lb_status lb_mlp_train(lb_mlp* m, int steps, float lr, float lr_min, float wd, float* losses) {
  if (!m || steps < 1 || m->n < 1 || !(lr > 0)) return LB_ERR_ARG;
  Sched sc = {0, steps, lr, lr_min, wd};
  MCK(cudaMemcpyAsync(m->sched, &sc, sizeof sc, cudaMemcpyHostToDevice, m->stream));
  if (!m->gexec) {
    MCK(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = train_step(m, m->cap);
    cudaGraph_t g = NULL;
    cudaError_t e2 = cudaStreamEndCapture(m->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&m->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return merr(m, "graph capture failed: %s", cudaGetErrorString(e)), LB_ERR_CUDA;
  }
  for (int i = 0; i < steps; ++i) MCK(cudaGraphLaunch(m->gexec, m->stream));
  if (losses) {
    // loss of the final parameters
    MCK(backward(m, m->stream));
    MCK(cudaMemcpyAsync(losses, m->loss, m->K * 4, cudaMemcpyDeviceToHost, m->stream));
  }
  MCK(cudaStreamSynchronize(m->stream));
  return LB_OK;
}

lb_status lb_mlp_predict(lb_mlp* m, int n, const float* x, float* mean, float* sd, float* members) {
  if (!m || n < 1 || !x || !mean || !sd) return LB_ERR_ARG;
  if (n > m->maxb) return merr(m, "batch larger than max_batch"), LB_ERR_ARG;
  float* dx = (float*)malloc_dev(m, (size_t)n * m->nin * 4 + 2 * (size_t)n * m->nout * 4);
  if (!dx) return merr(m, "device allocation failed"), LB_ERR_NOMEM;
  float* dmean = dx + (size_t)n * m->nin;
  float* dsd = dmean + (size_t)n * m->nout;
  MCK(cudaMemcpyAsync(dx, x, (size_t)n * m->nin * 4, cudaMemcpyHostToDevice, m->stream));
  pack_x_kernel<<<64, 256, 0, m->stream>>>(dx, n, m->nin, m->xbp);
  MCK(cudaGetLastError());
  MCK(forward(m, n, m->xbp, m->stream));
  ensemble_kernel<<<64, 256, 0, m->stream>>>(m->y, m->K, (long)m->maxb * m->nout, (long)n * m->nout, dmean, dsd);
  MCK(cudaGetLastError());
  MCK(cudaMemcpyAsync(mean, dmean, (size_t)n * m->nout * 4, cudaMemcpyDeviceToHost, m->stream));
  MCK(cudaMemcpyAsync(sd, dsd, (size_t)n * m->nout * 4, cudaMemcpyDeviceToHost, m->stream));
  if (members)
    for (int k = 0; k < m->K; ++k)
      MCK(cudaMemcpyAsync(members + (size_t)k * n * m->nout, m->y + (size_t)k * m->maxb * m->nout,
                          (size_t)n * m->nout * 4, cudaMemcpyDeviceToHost, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  if (m->have_alloc)
    m->alloc.free_fn(dx, (void*)m->stream, m->alloc.user);
  else
    cudaFree(dx);
  m->owned.pop_back();
  return LB_OK;
}

const char* lb_mlp_last_error(const lb_mlp* m) { return m ? m->err : g_mlp_err; }

}  // extern "C"
