// Separable transform solve of P1 on the tensor cores (3D grids, FP32_REFINED).
//
// Every 1D operator of P1 (Def. "def:operatorsP") is a Kronecker lift of D_2 (App. A.1), and on each
// axis D_2 with the boundary rule of Table "tab:bc" is diagonalised by an orthonormal transform:
//   Dirichlet axis (unknowns u = 1..N-1):       Q[k][u] = sqrt(2/N) sin(pi (k+1) u / N),
//   Neumann axis, even ghosts (u = 0..N-1):     Q[k][u] = sqrt(2/N) a_k cos(pi k (u + 1/2) / N), a_0 = 1/sqrt 2,
// with eigenvalues mu_k = 4 sin^2(pi k' / (2N)) of -h^2 D_aa (k' = k+1, resp. k).  Hence
//   6 h^2 P1 = (Qx (x) Qy (x) Qz)^T diag(6 c1 h^2 + 6 (mux + muy + muz) - (mux muy + muy muz + muz mux)) (Qx (x) Qy (x) Qz)
// and x = (6 h^2 P1)^{-1} b is three transforms, a pointwise scaling and three inverse transforms.
//
// Each transform along an axis is a dense GEMM D = Q X (Q: P x P, X: the field with the transformed
// axis as K), issued as tcgen05.mma (kind::f16, bf16 operands, FP32 accumulation in tensor memory)
// by one thread per CTA.  Three products hi*hi + hi*lo + lo*hi of the bf16 splits of Q and X give
// about 16 correct bits; the solve's result is then refined by Richardson sweeps with the exact
// residual (grid3d.cu), so the transform only has to be close, not exact.
//
// Operand layout in shared memory: K-major, no swizzle, 8 x 16-byte core matrices; core matrices
// adjacent in K are 128 bytes apart (leading byte offset), those adjacent in M / N 1024 bytes apart
// (stride byte offset), for K chunks of 64.  Each loader thread writes whole 16-byte core-matrix
// rows, eight consecutive threads one contiguous 128-byte run.
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "k_transform.cuh"

namespace ms {
namespace {

constexpr int TM = 128;                   // rows of the output tile (transform index)
constexpr int TN = 128;                   // data columns of the output tile
constexpr int KC = 64;                    // K per pipeline stage
constexpr int LBO = 128;                  // bytes between core matrices adjacent in K
constexpr int SBO = (KC / 8) * 128;       // bytes between core matrices adjacent in M / N
constexpr int TILE_BYTES = TM * KC * 2;   // one bf16 operand piece of a stage (TN == TM)
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // A hi, A lo, B hi, B lo
constexpr int GT = 512;                   // threads per CTA
constexpr int ITEMS = (TN * KC / 8) / GT; // B items (8 consecutive k of one column) per thread and chunk
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024;  // two stages, plus alignment slack
constexpr int kWaitTries = 1 << 20;       // bound of every mbarrier wait
static_assert(TN == TM, "operand pieces share one size");

__host__ __device__ inline int cm_off(int r, int k) { return (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets (all >> 4), the
// descriptor version of this architecture family (bit 46), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, N = TN, M = TM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(accumulate));
}

// Bounded wait for the phase of the given parity; false if it did not complete within the bound.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kWaitTries && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// 16-byte asynchronous copy global -> shared (completion by cp.async.wait_all).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Eight FP32 values to their bf16 hi parts and the bf16 rounding of the remainders.
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]), h1 = __float2bfloat16_rn(v[2 * e + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * e] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * e + 1] - __bfloat162float(h1));
    h[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// One transform pass over a P^3 array: out(m, n) = sum_k Q[m][k] in(k, n), element (k, n) of a
// tile at k sk + n1 sn1 + (n0b + j) sn0 for the tile's data columns n = n1 P + n0b + j.  Either the
// transformed axis is contiguous (sk == 1) or the data columns are (sn0 == 1).  mu != nullptr: the
// result is divided by the eigenvalue of 6 h^2 P1 at (m, n1, n0) (the last forward pass).
struct TsPass {
  const float* in;
  float* out;
  const uint4* qhi;  // A operand blocks [m tile][k chunk][TILE_BYTES], core-matrix layout
  const uint4* qlo;
  long long sk, sn1, sn0;
  int P, nkc;
  const float* mu_m;  // eigenvalue tables indexed by m, n1 and n0 (scaling pass only)
  const float* mu_1;
  const float* mu_0;
  float d6;
  int* err;
};

__global__ void __launch_bounds__(GT, 1) k_ts_gemm(TsPass p) {
  extern __shared__ unsigned char smraw[];
  unsigned char* const sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x;
  const long long n_start = (long long)blockIdx.y * TN;
  const long long n1 = n_start / p.P, n0b = n_start % p.P;
  const float* const inb = p.in + n1 * p.sn1 + n0b * p.sn0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // B item q of a chunk: column j and k group kg, placed so that eight consecutive threads write
  // one contiguous 128-byte run of a core-matrix column
  auto item = [&](int q, int& j, int& kg) {
    if (p.sk == 1) {
      j = (q >> 6) * 8 + (q & 7);
      kg = (q >> 3) & 7;
    } else {
      j = q & (TN - 1);
      kg = q / TN;
    }
  };
  // global loads of the B items of chunk c into registers
  auto load_b = [&](int c, float (&v)[ITEMS][8]) {
    const int k0 = c * KC;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      int j, kg;
      item(tid + GT * i, j, kg);
      if (p.sk == 1) {  // k contiguous: two 16-byte loads
        const float4* src = reinterpret_cast<const float4*>(inb + (long long)j * p.sn0 + k0 + kg * 8);
        const float4 a = src[0], b = src[1];
        v[i][0] = a.x; v[i][1] = a.y; v[i][2] = a.z; v[i][3] = a.w;
        v[i][4] = b.x; v[i][5] = b.y; v[i][6] = b.z; v[i][7] = b.w;
      } else {  // columns contiguous: a warp reads 32 consecutive columns of each k
        const float* src = inb + (long long)(k0 + kg * 8) * p.sk + j;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[i][e] = src[(long long)e * p.sk];
      }
    }
  };
  bool ok = true;
  int committed = 0;  // chunks whose MMAs were issued and committed
  float vb[ITEMS][8];
  load_b(0, vb);
  for (int c = 0; c < p.nkc; ++c) {
    const int s = c & 1;
    unsigned char* const st = sm + s * STAGE_BYTES;
    if (c >= 2) ok = mbar_wait(&mbar[s], ((c - 2) >> 1) & 1);  // the MMAs that last read this stage
    ok = __syncthreads_and(ok);  // one decision for the whole block
    if (!ok) break;
    // A: the transform matrix block, already in the operand layout, copied asynchronously
    const uint4* qh = p.qhi + (size_t)(mt * p.nkc + c) * (TILE_BYTES / 16);
    const uint4* ql = p.qlo + (size_t)(mt * p.nkc + c) * (TILE_BYTES / 16);
#pragma unroll
    for (int i = tid; i < TILE_BYTES / 16; i += GT) {
      cp_async16(st + 16 * i, qh + i);
      cp_async16(st + TILE_BYTES + 16 * i, ql + i);
    }
    // B of this chunk (in registers) split into bf16 hi / lo core-matrix rows
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      int j, kg;
      item(tid + GT * i, j, kg);
      uint4 hi, lo;
      split8(vb[i], hi, lo);
      const int off = cm_off(j, kg * 8);
      *reinterpret_cast<uint4*>(st + 2 * TILE_BYTES + off) = hi;
      *reinterpret_cast<uint4*>(st + 3 * TILE_BYTES + off) = lo;
    }
    if (c + 1 < p.nkc) load_b(c + 1, vb);  // in flight during the MMAs of this chunk
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(st), a_lo = a_hi + TILE_BYTES;
      const uint32_t b_hi = a_hi + 2 * TILE_BYTES, b_lo = a_hi + 3 * TILE_BYTES;
#pragma unroll
      for (int kk = 0; kk < KC / 16; ++kk) {
        const uint32_t ko = kk * 2 * LBO;  // 16 elements of K = two core matrices
        mma_bf16(tmem, smem_desc(a_lo + ko), smem_desc(b_hi + ko), (c > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(tmem, smem_desc(a_hi + ko), smem_desc(b_lo + ko), 1u);
        mma_bf16(tmem, smem_desc(a_hi + ko), smem_desc(b_hi + ko), 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[s]))
                   : "memory");
    }
    committed = c + 1;
  }
  // the last commit covers every MMA issued before it; after a timeout it is waited for once more
  // (bounded), so that no MMA is in flight when the tensor memory is released
  bool drained = true;
  if (committed > 0) {
    const int cl = committed - 1;
    drained = mbar_wait(&mbar[cl & 1], (cl >> 1) & 1);
  }
  ok = __syncthreads_and(ok && drained);
  if (!ok) {
    if (tid == 0) atomicExch(p.err, 1);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warp w: tensor-memory lanes (rows) 32 (w % 4) .., columns 32 (w / 4) .. + 31
    const int m = mt * TM + 32 * (warp & 3) + lane;
    const int jb = 32 * (warp >> 2);
    float* const outb = p.out + (long long)m * p.sk + n1 * p.sn1 + n0b * p.sn0;
    float mum = 0.0f, mu1 = 0.0f;
    if (p.mu_m) {
      mum = p.mu_m[m];
      mu1 = p.mu_1[n1];
    }
#pragma unroll
    for (int cc = 0; cc < 32; cc += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(jb + cc)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float y[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        y[e] = __uint_as_float(r[e]);
        if (p.mu_m) {
          const float mu0 = p.mu_0[n0b + jb + cc + e];
          const float eig = p.d6 + 6.0f * ((mum + mu1) + mu0) - ((mum * mu1 + mu1 * mu0) + mu0 * mum);
          y[e] = y[e] / eig;
        }
      }
      if (p.sn0 == 1) {
        float4* o = reinterpret_cast<float4*>(outb + jb + cc);
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = make_float4(y[4 * e], y[4 * e + 1], y[4 * e + 2], y[4 * e + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) outb[(long long)(jb + cc + e) * p.sn0] = y[e];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

// The unknowns of a component (axis a: first unknown u0[a], count nu[a]) into the P^3 working array
// [z][y][x], zero on the padding.
__global__ void k_ts_pack(const float* __restrict__ b, Shape3 s, float* __restrict__ w, int P, int3 u0, int3 nu) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= P) return;
  float v = 0.0f;
  if (x < nu.x && y < nu.y && z < nu.z)
    v = b[((size_t)(z + u0.z) * s.n[1] + (y + u0.y)) * s.n[0] + (x + u0.x)];
  w[((size_t)z * P + y) * P + x] = v;
}

// The working array back into a component's layout; wall points (not unknowns) get zero.
__global__ void k_ts_unpack(const float* __restrict__ w, Shape3 s, float* __restrict__ xo, int P, int3 u0, int3 nu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= s.n[0]) return;
  const int x = i - u0.x, y = j - u0.y, z = k - u0.z;
  float v = 0.0f;
  if (x >= 0 && x < nu.x && y >= 0 && y < nu.y && z >= 0 && z < nu.z) v = w[((size_t)z * P + y) * P + x];
  xo[((size_t)k * s.n[1] + j) * s.n[0] + i] = v;
}

// Transform matrix of a boundary type (DIR: sine, NEU: cosine), orthonormal on its nu unknowns,
// embedded in P x P with zeros; mu: its eigenvalues of -h^2 D_aa (0 on the padding).
void transform_matrix(int N, int P, int bc, std::vector<double>* Q, std::vector<double>* mu) {
  Q->assign((size_t)P * P, 0.0);
  mu->assign(P, 0.0);
  const int nu = bc == DIR ? N - 1 : N;
  const double c = std::sqrt(2.0 / N);
  for (int k = 0; k < nu; ++k) {
    const int kk = bc == DIR ? k + 1 : k;
    const double sk = std::sin(M_PI * kk / (2.0 * N));
    (*mu)[k] = 4.0 * sk * sk;
    for (int u = 0; u < nu; ++u) {
      double v;
      if (bc == DIR) {
        // sin(pi kk (u+1) / N), argument reduced exactly in integers
        const long q = ((long)kk * (u + 1)) % (2L * N);
        v = c * std::sin(M_PI * (double)q / N);
      } else {
        const long q = ((long)kk * (2L * u + 1)) % (4L * N);
        v = c * (k == 0 ? std::sqrt(0.5) : 1.0) * std::cos(M_PI * (double)q / (2.0 * N));
      }
      (*Q)[(size_t)k * P + u] = v;
    }
  }
}

// A = M (or its transpose) as bf16 hi / lo operand blocks [m tile][k chunk] in the core-matrix layout.
void operand_blocks(const std::vector<double>& M, int P, bool transpose, std::vector<uint16_t>* hi,
                    std::vector<uint16_t>* lo) {
  const int nmt = P / TM, nkc = P / KC;
  hi->assign((size_t)P * P, 0);
  lo->assign((size_t)P * P, 0);
  for (int mt = 0; mt < nmt; ++mt)
    for (int kc = 0; kc < nkc; ++kc) {
      uint16_t* bh = hi->data() + (size_t)(mt * nkc + kc) * (TILE_BYTES / 2);
      uint16_t* bl = lo->data() + (size_t)(mt * nkc + kc) * (TILE_BYTES / 2);
      for (int r = 0; r < TM; ++r)
        for (int k = 0; k < KC; ++k) {
          const int m = mt * TM + r, kk = kc * KC + k;
          const double v = transpose ? M[(size_t)kk * P + m] : M[(size_t)m * P + kk];
          const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
          const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
          bh[cm_off(r, k) / 2] = __bfloat16_as_ushort(h);
          bl[cm_off(r, k) / 2] = __bfloat16_as_ushort(l);
        }
    }
}

}  // namespace

int ts_setup(int N, TransformSolver* ts, std::string* err) {
  ts->N = N;
  ts->P = ((N + TM - 1) / TM) * TM;
  const int P = ts->P;
  const size_t n3 = (size_t)P * P * P;
  if (cudaFuncSetAttribute(k_ts_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess) {
    *err = "cannot configure shared memory of the transform GEMM";
    return -1;
  }
  for (int k = 0; k < 2; ++k)
    if (dev_malloc(&ts->w[k], n3 * sizeof(float)) != cudaSuccess) {
      *err = "cudaMalloc of the transform working arrays failed";
      return -2;
    }
  if (dev_malloc(&ts->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ts->d_err, 0, sizeof(int)) != cudaSuccess) {
    *err = "cudaMalloc of the transform error flag failed";
    return -2;
  }
  for (int bc = 0; bc < 2; ++bc) {
    std::vector<double> Q, mu;
    transform_matrix(N, P, bc, &Q, &mu);
    std::vector<float> muf(mu.begin(), mu.end());
    if (dev_malloc(&ts->mu[bc], P * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(ts->mu[bc], muf.data(), P * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      *err = "transform eigenvalue tables failed";
      return -2;
    }
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<uint16_t> hi, lo;
      operand_blocks(Q, P, dir == 1, &hi, &lo);
      for (int part = 0; part < 2; ++part) {
        const std::vector<uint16_t>& v = part ? lo : hi;
        if (dev_malloc(&ts->q[bc][dir][part], v.size() * 2) != cudaSuccess ||
            cudaMemcpy(ts->q[bc][dir][part], v.data(), v.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
          *err = "transform matrices failed";
          return -2;
        }
      }
    }
  }
  return 0;
}

void ts_free(TransformSolver* ts) {
  for (float* p : ts->w) dev_free(p);
  for (auto& a : ts->q)
    for (auto& b : a)
      for (uint4* p : b) dev_free(p);
  for (float* p : ts->mu) dev_free(p);
  dev_free(ts->d_err);
  *ts = TransformSolver{};
}

int ts_solve(const TransformSolver& ts, const Shape3& s, const float* b, float* x, float d6, cudaStream_t st,
             ms_grid* g) {
  const int P = ts.P;
  const long long P2 = (long long)P * P;
  int3 u0, nu;
  const int bc[3] = {s.bc[0], s.bc[1], s.bc[2]};
  u0.x = bc[0] == DIR ? 1 : 0;
  u0.y = bc[1] == DIR ? 1 : 0;
  u0.z = bc[2] == DIR ? 1 : 0;
  nu.x = bc[0] == DIR ? ts.N - 1 : ts.N;
  nu.y = bc[1] == DIR ? ts.N - 1 : ts.N;
  nu.z = bc[2] == DIR ? ts.N - 1 : ts.N;
  const double n3 = (double)P2 * P;
  k_ts_pack<<<dim3((P + 127) / 128, P, P), 128, 0, st>>>(b, s, ts.w[0], P, u0, nu);
  prof_mark(g, KK_TSPACK, 4.0 * (double)s.size() + 4.0 * n3);
  // (sk, sn1, sn0) of a pass along x, y, z over the [z][y][x] working array
  const long long strides[3][3] = {{1, P2, P}, {P, P2, 1}, {P2, P, 1}};
  const dim3 grid(P / TM, (unsigned)(P2 / TN));
  int cur = 0, launches = 1;
  auto pass = [&](int axis, int dir, bool scale) {
    TsPass p;
    p.in = ts.w[cur];
    p.out = ts.w[cur ^ 1];
    p.qhi = ts.q[bc[axis]][dir][0];
    p.qlo = ts.q[bc[axis]][dir][1];
    p.sk = strides[axis][0];
    p.sn1 = strides[axis][1];
    p.sn0 = strides[axis][2];
    p.P = P;
    p.nkc = P / KC;
    // scaling pass (along z): m = kz, n1 = ky, n0 = kx
    p.mu_m = scale ? ts.mu[bc[2]] : nullptr;
    p.mu_1 = scale ? ts.mu[bc[1]] : nullptr;
    p.mu_0 = scale ? ts.mu[bc[0]] : nullptr;
    p.d6 = d6;
    p.err = ts.d_err;
    k_ts_gemm<<<grid, GT, SMEM_BYTES, st>>>(p);
    prof_mark(g, KK_TSGEMM, 8.0 * n3);  // the working array read and written once
    cur ^= 1;
    ++launches;
  };
  pass(0, 0, false);
  pass(1, 0, false);
  pass(2, 0, true);
  pass(2, 1, false);
  pass(1, 1, false);
  pass(0, 1, false);
  k_ts_unpack<<<dim3((s.n[0] + 127) / 128, s.n[1], s.n[2]), 128, 0, st>>>(ts.w[cur], s, x, P, u0, nu);
  prof_mark(g, KK_TSPACK, 4.0 * n3 + 4.0 * (double)s.size());
  return launches + 1;
}

}  // namespace ms
