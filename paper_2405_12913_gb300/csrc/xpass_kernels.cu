// The x-pass of the split Poisson solve: with the density transformed over (y, z) by batched 2D cuFFT plans, one
// kernel does, per pencil (ky, kz) along x, the forward x-FFT, the fused k-space step (Green's function of the
// Poisson equation of Sec. 2, derivative i k_j, per-axis deconvolution and smoothing, learned factor g) and the
// inverse x-FFTs of the gradient spectra; batched 2D C2R plans finish the gradient fields.  Together with the 2D
// plans this reads and writes every spectrum once less than a 3D R2C, a separate k-space kernel and 3D C2Rs.
//
// Tiles.  The [x][ky][kz] half spectrum (kz rows of n/2 + 1 complex values, as cuFFT writes them) is viewed as n
// x-planes of F = n (n/2 + 1) consecutive (ky, kz) pencils.  A tile is TK = 8P consecutive pencils of that flat
// index for all n x-planes: TK x 8 bytes per plane (64 B at n = 1024), which start on a 64-byte boundary in every
// plane because F is a multiple of TK.  So a tile is one 2D box of a TMA tensor map (inner extent the flat
// index, outer extent x), with no padding of the rows that cuFFT reads and writes, and every tile is full.  A
// tile may span two ky rows; each pencil takes its own (ky, kz).
//
// Data movement.  Input tiles arrive by TMA (cp.async.bulk.tensor) into one of two shared buffers, completing on
// an mbarrier; the next tile is requested while the current one is transformed.  Outputs are written row-wise
// into a staging buffer and leave by TMA stores (bulk groups), so that no thread issues a global load or store
// per element.  The buffers carry the TMA swizzle (64 B or 128 B), which spreads a pencil's column over 8 of the
// 16 eight-byte bank slots of a 128-byte line.
//
// FFT along x (n = 32 R1 points), four-step with x = l + 32 m and k = k1 + R1 k2.  A warp owns P = 32 / R1
// pencils.  Lane l first holds x = l + 32 m of its P pencils (its column of the tile), does the R1-point DFTs
// over m in registers and applies the twiddles W_n^(l k1); a transpose through the warp's private 8 KB of the
// (already read) input buffer gives lane (p, k1) the 32 values over l, and a 32-point DFT over l in registers
// leaves X[k1 + R1 k2] of pencil p in that lane.  The inverse runs the same steps backwards.  The gradient
// spectra are linear in the pencil: for a pencil (ky, kz) the y and z components are d_y V and d_z V with
// V = IFFT_x(i c X), so a filter set needs two inverse transforms (V and the x component) for its three outputs.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "common.h"
#include "tma.h"
#include "xpass.h"

namespace hrt {

namespace {

constexpr int kXWarps = 8;
constexpr int kXThreads = kXWarps * 32;
constexpr int kTileBytes = 64 * 1024;  // TK pencils x n rows x 8 bytes, for every supported n
// Bounded waits (tma::mbar_wait): after about a second the kernel records kXpassTimeout and returns.
using namespace tma;

__host__ __device__ constexpr int bit_reverse(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// (cos, sin) of 2 pi t / 32, t in [0, 16): FP64 values rounded to float.
__device__ __forceinline__ float2 cs32(int t) {
  switch (t) {
    case 1: return make_float2(9.807852804e-01f, 1.950903220e-01f);
    case 2: return make_float2(9.238795325e-01f, 3.826834324e-01f);
    case 3: return make_float2(8.314696123e-01f, 5.555702330e-01f);
    case 4: return make_float2(7.071067812e-01f, 7.071067812e-01f);
    case 5: return make_float2(5.555702330e-01f, 8.314696123e-01f);
    case 6: return make_float2(3.826834324e-01f, 9.238795325e-01f);
    case 7: return make_float2(1.950903220e-01f, 9.807852804e-01f);
    case 9: return make_float2(-1.950903220e-01f, 9.807852804e-01f);
    case 10: return make_float2(-3.826834324e-01f, 9.238795325e-01f);
    case 11: return make_float2(-5.555702330e-01f, 8.314696123e-01f);
    case 12: return make_float2(-7.071067812e-01f, 7.071067812e-01f);
    case 13: return make_float2(-8.314696123e-01f, 5.555702330e-01f);
    case 14: return make_float2(-9.238795325e-01f, 3.826834324e-01f);
    case 15: return make_float2(-9.807852804e-01f, 1.950903220e-01f);
    default: return make_float2(1.f, 0.f);
  }
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// b * W_32^(+-t): the forward kernel exp(-2 pi i t / 32), the inverse its conjugate; t = 0 and the quarter turn
// t = 8 without multiplications.
template <bool INV>
__device__ __forceinline__ float2 twiddle32(float2 b, int t) {
  if (t == 0) return b;
  if (t == 8) return INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
  const float2 w = cs32(t);
  return INV ? make_float2(b.x * w.x - b.y * w.y, b.x * w.y + b.y * w.x)
             : make_float2(b.x * w.x + b.y * w.y, b.y * w.x - b.x * w.y);
}

// In-register radix-2 DFT of N <= 32 points v[OFF .. OFF + N) (natural order in and out, unnormalised).  The
// stage loop counts stages (not a shifted length) so that it unrolls fully and v stays in registers.
template <int N, bool INV, int OFF>
__device__ __forceinline__ void dft(float2 (&v)[32]) {
  constexpr int kBits = ilog2(N);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = bit_reverse(i, kBits);
    if (j > i) {
      const float2 t = v[OFF + i];
      v[OFF + i] = v[OFF + j];
      v[OFF + j] = t;
    }
  }
#pragma unroll
  for (int st = 0; st < kBits; ++st) {
    const int half = 1 << st, len = 2 << st;
#pragma unroll
    for (int grp = 0; grp < N / 2; ++grp) {
      const int i = (grp >> st) * len, k = grp & (half - 1);
      const float2 a = v[OFF + i + k];
      const float2 b = twiddle32<INV>(v[OFF + i + k + half], k * (32 / len));
      v[OFF + i + k] = cadd(a, b);
      v[OFF + i + k + half] = csub(a, b);
    }
  }
}

// The R1-point DFTs of all P pencils of a lane (layout A), with compile-time register offsets.
template <int R1, bool INV, int P>
struct DftPencils {
  __device__ __forceinline__ static void run(float2 (&v)[32]) {
    dft<R1, INV, (P - 1) * R1>(v);
    DftPencils<R1, INV, P - 1>::run(v);
  }
};
template <int R1, bool INV>
struct DftPencils<R1, INV, 0> {
  __device__ __forceinline__ static void run(float2 (&)[32]) {}
};

// ---- shared memory, mbarriers and TMA (inline PTX) -------------------------------------------------------

// ---- tile geometry ----------------------------------------------------------------------------------------
// TK = 8P pencils per tile; the tile is stored as NSUB sub-tiles of SUBW columns (rows of PITCH = 8 SUBW bytes,
// at most 128 so that a TMA swizzle applies): element (row r, column c) sits at sub-tile c / SUBW, row r,
// 8-byte slot c % SUBW, with the 16-byte chunk index XORed by the swizzle key of the row.
template <int R1>
struct Geo {
  static constexpr int P = 32 / R1;
  static constexpr int N = 32 * R1;
  static constexpr int TK = kXWarps * P;
  static constexpr int SUBW = TK < 16 ? TK : 16;
  static constexpr int NSUB = TK / SUBW;
  static constexpr int PITCH = SUBW * 8;
  static constexpr int SUB_BYTES = N * PITCH;
  static constexpr int ROWS_PER_BOX = N < 256 ? N : 256;
  static constexpr int BOXES = N / ROWS_PER_BOX;
  static_assert(TK * N * 8 == kTileBytes, "a tile is 64 KB");
  // Swizzle key of row r: address bits [7, 9) (64 B pitch, SWIZZLE_64B) or [7, 10) (128 B, SWIZZLE_128B).
  __device__ __forceinline__ static int key(int r) { return PITCH == 64 ? (r >> 1) & 3 : r & 7; }
  // Byte offset of (r, c) within the tile.
  __device__ __forceinline__ static int offset(int r, int c) {
    const int sub = c / SUBW, cc = c - sub * SUBW;
    return sub * SUB_BYTES + r * PITCH + ((cc * 8) ^ (key(r) << 4));
  }
};

struct Pencil {
  int ky, kz;
};

__device__ __forceinline__ float learned_factor(const XpassSet& s, float kmag) {
  if (s.g == nullptr) return 1.f;
  const float t = kmag * s.g_inv_dk;
  if (t >= static_cast<float>(s.g_nk - 1)) return 1.f;
  const int i = static_cast<int>(t);
  const float w = t - static_cast<float>(i);
  return __ldg(s.g + i) * (1.f - w) + __ldg(s.g + i + 1) * w;
}

__device__ __forceinline__ float dx_of(int kx, int n, float kf) {
  const int nx = kx < (n >> 1) ? kx : kx - n;
  return nx == -(n >> 1) ? 0.f : kf * nx;
}

// u[k2] = d(kx) Y[k2] at kx = k1 + R1 k2, with Y = i c X, c = Green's function x per-axis filter factors x learned
// g (the k-space kernel's factor): computed here from X (PRE false) or already in X (PRE true); d = d_x of each
// kx for the x component, else 1.
template <int R1, bool PRE>
__device__ __forceinline__ void filtered(const float2 (&X)[32], float2 (&u)[32], const XpassSet& s,
                                         const float* wx, int k1, float kf, float scale, float k2yz, float cyz,
                                         bool with_dx) {
  constexpr int N = 32 * R1;
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) {
    const int kx = k1 + R1 * k2;
    const float d = with_dx ? dx_of(kx, N, kf) : 1.f;
    if (PRE) {
      u[k2] = make_float2(d * X[k2].x, d * X[k2].y);
    } else {
      const int nx = kx < (N >> 1) ? kx : kx - N;
      const float kxf = kf * nx;
      const float kk = kxf * kxf + k2yz;
      float c = kk > 0.f ? __fdividef(scale, kk) : 0.f;
      c *= wx[kx] * cyz;
      if (s.g != nullptr) c *= learned_factor(s, sqrtf(kk));
      c *= d;
      u[k2] = make_float2(-c * X[k2].y, c * X[k2].x);
    }
  }
}

// The warp's private transpose area: 32 rows q of 32 complex values, slot (q, l) at q * 32 + (l ^ q) (an XOR
// that keeps both the row-wise writes and the column-wise reads of a warp on 16 distinct 8-byte slots).
__device__ __forceinline__ float2* tslot(char* priv, int q, int l) {
  return reinterpret_cast<float2*>(priv + q * 256 + ((l ^ q) << 3));
}

// Inverse x-FFT from layout B (lane (p, k1), u[k2] = X[k1 + R1 k2]) to layout A (lane l, u[p R1 + n2] =
// x[l + 32 n2]) through the warp's private area.
template <int R1>
__device__ __forceinline__ void inverse_x(float2 (&u)[32], char* priv, const float2* twi, int lane) {
  constexpr int P = 32 / R1;
  dft<32, true, 0>(u);
#pragma unroll
  for (int n1 = 1; n1 < 32; ++n1) u[n1] = cmul(u[n1], twi[n1 * 32 + lane]);
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) *tslot(priv, lane, n1) = u[n1];
  __syncwarp();
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int j = 0; j < R1; ++j) u[p * R1 + j] = *tslot(priv, p * R1 + j, lane);
  __syncwarp();
  DftPencils<R1, true, P>::run(u);
}

// Pencil frequencies and the per-pencil factors of one filter set.
struct PencilFactors {
  float k2yz, cyz, dy, dz;
};

__device__ __forceinline__ PencilFactors pencil_factors(const XpassSet& s, Pencil pc, int n, float kf) {
  const int half = n >> 1;
  const int ny = pc.ky < half ? pc.ky : pc.ky - n;
  const float kyf = kf * ny, kzf = kf * pc.kz;
  PencilFactors f;
  f.k2yz = kyf * kyf + kzf * kzf;
  f.cyz = __ldg(s.wxy + pc.ky) * __ldg(s.wz + pc.kz);
  f.dy = ny == -half ? 0.f : kyf;
  f.dz = pc.kz == half ? 0.f : kzf;
  return f;
}

template <int R1, bool TWO>
__global__ void __launch_bounds__(kXThreads, 1)
    xpass_kernel(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ CUtensorMap out_a,
                 const __grid_constant__ CUtensorMap out_b, int nzc, int n_tiles, float kf, float scale,
                 const float2* __restrict__ tw, XpassSet a, XpassSet b, int* __restrict__ err,
                 float4* __restrict__ clear, int64_t clear_n4, int64_t clear_per) {
  using G = Geo<R1>;
  constexpr int P = G::P, N = G::N, TK = G::TK;
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned base: the 128-byte swizzle repeats every 1024 bytes and is taken from address bits
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* const ibuf0 = sm;
  unsigned char* const ibuf1 = sm + kTileBytes;
  unsigned char* const obuf = sm + 2 * kTileBytes;
  float2* twf = reinterpret_cast<float2*>(sm + 3 * kTileBytes);  // [R1][32]: W_n^(l k1)
  float2* twi = twf + R1 * 32;                                     // [32][32]: W_n^(-n1 k1(lane))
  float* wxa = reinterpret_cast<float*>(twi + 32 * 32);
  float* wxb = wxa + N;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wxb + N);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < R1 * 32 + 32 * 32; i += kXThreads) twf[i] = tw[i];
  for (int i = tid; i < N; i += kXThreads) {
    wxa[i] = __ldg(a.wxy + i);
    wxb[i] = TWO ? __ldg(b.wxy + i) : 0.f;
  }
  const uint32_t bar0 = smem_u32(bars), bar1 = smem_u32(bars + 1);
  const uint32_t ib0 = smem_u32(ibuf0), ib1 = smem_u32(ibuf1), ob = smem_u32(obuf);
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    fence_mbar_init();
  }
  __syncthreads();

  // one thread requests tile t into the input buffer at dst
  auto request = [&](int t, uint32_t dst, uint32_t bar) {
    mbar_expect_tx(bar, kTileBytes);
#pragma unroll
    for (int s = 0; s < G::NSUB; ++s)
#pragma unroll
      for (int bx = 0; bx < G::BOXES; ++bx)
        load_2d(dst + s * G::SUB_BYTES + bx * G::ROWS_PER_BOX * G::PITCH, &in_map,
                    2 * (t * TK + s * G::SUBW), bx * G::ROWS_PER_BOX, bar);
  };
  // one thread stores the staged tile at src as component comp of the set's output spectra
  auto store = [&](const CUtensorMap* map, uint32_t src, int t, int comp) {
#pragma unroll
    for (int s = 0; s < G::NSUB; ++s)
#pragma unroll
      for (int bx = 0; bx < G::BOXES; ++bx)
        store_3d(map, src + s * G::SUB_BYTES + bx * G::ROWS_PER_BOX * G::PITCH, 2 * (t * TK + s * G::SUBW),
                     bx * G::ROWS_PER_BOX, comp);
  };

  // loads requested and not yet consumed, one bit per input buffer (thread 0's bookkeeping, for the exit after
  // a timed-out wait)
  uint32_t pending = 0u;
  if (tid == 0 && static_cast<int>(blockIdx.x) < n_tiles) {
    request(blockIdx.x, ib0, bar0);
    pending = 1u;
  }
  const int col0 = warp * P;
  const int pp = lane / R1, k1 = lane - pp * R1;
  // per-lane byte offsets of the warp's columns at rows lane + 32 m (the swizzle key depends on lane only)
  int coff[P];
#pragma unroll
  for (int p = 0; p < P; ++p) coff[p] = G::offset(lane, col0 + p);
  uint32_t parity = 0u;  // bit c: the phase parity to wait for on input buffer c
  int k = 0;
  bool ok = true;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
    if (clear) {
      // this tile's slice of a dead buffer (the density the 2D R2C has consumed), zeroed for the next deposit
      // while the tile's copy is in flight: plain 16-byte stores of consecutive addresses, which the pass's
      // spare DRAM bandwidth absorbs
      const int64_t lo = static_cast<int64_t>(tile) * clear_per;
      const int64_t hi = lo + clear_per < clear_n4 ? lo + clear_per : clear_n4;
      for (int64_t i = lo + tid; i < hi; i += kXThreads) clear[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int cb = k & 1;
    unsigned char* const ib = cb ? ibuf1 : ibuf0;
    const uint32_t ibs = cb ? ib1 : ib0;
    const bool got = mbar_wait(cb ? bar1 : bar0, (parity >> cb) & 1u);
    parity ^= 1u << cb;
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    pending &= ~(1u << cb);
    // ---- the warp's columns: X[p R1 + m] = x[lane + 32 m] of pencil col0 + p
    float2 X[32];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int m = 0; m < R1; ++m)
        X[p * R1 + m] = *reinterpret_cast<const float2*>(ib + coff[p] + m * 32 * G::PITCH);
    __syncthreads();  // every column read: the input buffer is now the warps' transpose area
    char* const priv = reinterpret_cast<char*>(ib) + warp * 8192;
    // ---- forward x-FFT: X[k2] = spectrum at kx = k1 + R1 k2 of pencil col0 + pp
    DftPencils<R1, false, P>::run(X);
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int j = 1; j < R1; ++j) X[p * R1 + j] = cmul(X[p * R1 + j], twf[j * 32 + lane]);
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int j = 0; j < R1; ++j) *tslot(priv, p * R1 + j, lane) = X[p * R1 + j];
    __syncwarp();
#pragma unroll
    for (int l = 0; l < 32; ++l) X[l] = *tslot(priv, lane, l);
    __syncwarp();
    dft<32, false, 0>(X);

    // this lane's pencil in layout B, and the warp's P pencils in layout A (for the d_y, d_z scaling)
    const int flat0 = tile * TK + col0;
    const int fb = flat0 + pp;
    const Pencil pb{fb / nzc, fb - (fb / nzc) * nzc};
    const PencilFactors fa_b = pencil_factors(a, pb, N, kf);
    if (!TWO) {
      // one filter set: Y = i c X once, in place
      float2 u[32];
      filtered<R1, false>(X, u, a, wxa, k1, kf, scale, fa_b.k2yz, fa_b.cyz, false);
#pragma unroll
      for (int i = 0; i < 32; ++i) X[i] = u[i];
    }
    // ---- inverse transforms: per set, the x component, then V (stored as d_y V and d_z V)
    constexpr int kOutputs = TWO ? 4 : 2;
#pragma unroll 1
    for (int w = 0; w < kOutputs; ++w) {
      const bool second = TWO && w >= 2;
      const XpassSet& s = second ? b : a;
      const bool xcomp = (w & 1) == 0;
      float2 u[32];
      if (TWO) {
        const PencilFactors f = second ? pencil_factors(b, pb, N, kf) : fa_b;
        filtered<R1, false>(X, u, s, second ? wxb : wxa, k1, kf, scale, f.k2yz, f.cyz, xcomp);
      } else {
        filtered<R1, true>(X, u, s, wxa, k1, kf, scale, 0.f, 0.f, xcomp);
      }
      inverse_x<R1>(u, priv, twi, lane);
      // staging: every earlier store has read its source, and every warp is done with its transposes
      if (tid == 0) bulk_wait_read_all();
      __syncthreads();
      if (tid == 0 && w == 0) {
        // the other input buffer's last reader (the previous tile's stores) is done: request the next tile
        const int next = tile + gridDim.x;
        if (next < n_tiles) {
          fence_async_shared();
          request(next, cb ? ib0 : ib1, cb ? bar0 : bar1);
          pending |= 1u << (cb ^ 1);
        }
      }
      const CUtensorMap* map = second ? &out_b : &out_a;
      if (xcomp) {
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
          for (int m = 0; m < R1; ++m)
            *reinterpret_cast<float2*>(obuf + coff[p] + m * 32 * G::PITCH) = u[p * R1 + m];
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
          store(map, ob, tile, 0);
          bulk_commit();
        }
      } else {
        // d_y V into the staging buffer, d_z V (three outputs) into the input buffer, whose transposes are done
        const bool with_z = s.n_out == 3;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int f = flat0 + p;
          const Pencil pc{f / nzc, f - (f / nzc) * nzc};
          const PencilFactors pf = pencil_factors(s, pc, N, kf);
#pragma unroll
          for (int m = 0; m < R1; ++m) {
            const float2 v = u[p * R1 + m];
            *reinterpret_cast<float2*>(obuf + coff[p] + m * 32 * G::PITCH) = make_float2(pf.dy * v.x, pf.dy * v.y);
            if (with_z)
              *reinterpret_cast<float2*>(ib + coff[p] + m * 32 * G::PITCH) = make_float2(pf.dz * v.x, pf.dz * v.y);
          }
        }
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
          store(map, ob, tile, 1);
          if (with_z) store(map, ibs, tile, 2);
          bulk_commit();
        }
        if (TWO && !second) {
          // set b transposes through the input buffer again: wait until its d_z V store has read it
          if (tid == 0) bulk_wait_read_all();
          __syncthreads();
        }
      }
    }
  }
  if (tid == 0) {
    bulk_wait_all();
    if (!ok) {
      atomicOr(err, kXpassTimeout);
      // let requested loads land before the block's shared memory goes away (again a bounded wait); the
      // timed-out buffer's parity was already advanced
      for (int c = 0; c < 2; ++c)
        if ((pending >> c) & 1u) mbar_wait(c ? bar1 : bar0, ((parity >> c) & 1u) ^ (c == (k & 1) ? 1u : 0u));
    }
  }
}

}  // namespace

hrt_status tensor_map_encoder(EncodeTiled* out) {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q{};
    void* p = nullptr;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = reinterpret_cast<EncodeTiled>(p);
  });
  if (!fn) return cuda_status(e == cudaSuccess ? cudaErrorSymbolNotFound : e, "cuTensorMapEncodeTiled entry point");
  *out = fn;
  return HRT_OK;
}

namespace {

// Tensor map over the [comp][x][flat pencil] spectra: rank 2 (one spectrum) or 3; boxes of (2 SUBW floats) x
// (rows per box) x 1.
template <int R1>
hrt_status make_map(CUtensorMap* map, const void* base, int n, int comps) {
  using G = Geo<R1>;
  EncodeTiled enc = nullptr;
  HRT_TRY(tensor_map_encoder(&enc));
  const uint64_t flat = static_cast<uint64_t>(n) * (n / 2 + 1);
  const cuuint64_t dims[3] = {2 * flat, static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(comps)};
  const cuuint64_t strides[2] = {flat * sizeof(float2), flat * sizeof(float2) * n};
  const cuuint32_t box[3] = {2 * G::SUBW, G::ROWS_PER_BOX, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, comps > 0 ? 3 : 2, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         G::PITCH == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HRT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return HRT_OK;
}

}  // namespace

bool xpass_supported(int64_t n) { return n == 256 || n == 512 || n == 1024; }

int64_t xpass_row(int64_t n) { return n / 2 + 1; }

void xpass_twiddles(int64_t n, std::vector<float2>& tw) {
  const int r1 = static_cast<int>(n / 32);
  tw.assign(static_cast<size_t>(r1) * 32 + 32 * 32, make_float2(0.f, 0.f));
  const double two_pi = 2.0 * M_PI;
  for (int k1 = 0; k1 < r1; ++k1)
    for (int l = 0; l < 32; ++l) {
      const double ph = -two_pi * static_cast<double>((static_cast<int64_t>(l) * k1) % n) / static_cast<double>(n);
      tw[k1 * 32 + l] = make_float2(static_cast<float>(std::cos(ph)), static_cast<float>(std::sin(ph)));
    }
  for (int n1 = 0; n1 < 32; ++n1)
    for (int t = 0; t < 32; ++t) {
      const int k1 = t % r1;
      const double ph = two_pi * static_cast<double>((static_cast<int64_t>(n1) * k1) % n) / static_cast<double>(n);
      tw[r1 * 32 + n1 * 32 + t] = make_float2(static_cast<float>(std::cos(ph)), static_cast<float>(std::sin(ph)));
    }
}

size_t xpass_smem_bytes(int64_t n) {
  const size_t r1 = static_cast<size_t>(n / 32);
  return 1024 + 3 * static_cast<size_t>(kTileBytes) + (r1 * 32 + 32 * 32) * sizeof(float2) +
         2 * static_cast<size_t>(n) * sizeof(float) + 2 * sizeof(uint64_t);
}

template <int R1, bool TWO>
static hrt_status launch_r1(const void* in, int64_t n, double box, double pref, const float2* tw,
                            const XpassSet& a, const XpassSet& b, int* err, float* clear, int64_t clear_floats,
                            cudaStream_t s) {
  using G = Geo<R1>;
  const int nzc = static_cast<int>(n / 2 + 1);
  const int64_t flat = n * nzc;
  if (flat % G::TK != 0) return fail(HRT_ERR_INVALID_ARG, "x-pass: pencils per plane not a multiple of the tile");
  for (const XpassSet* x : {&a, &b})
    if (x->n_out > 0 && (reinterpret_cast<uintptr_t>(x->out) & 15) != 0)
      return fail(HRT_ERR_INVALID_ARG, "x-pass: output spectra must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(in) & 15) != 0) return fail(HRT_ERR_INVALID_ARG, "x-pass: input must be 16-byte aligned");
  if (clear && ((reinterpret_cast<uintptr_t>(clear) & 15) != 0 || clear_floats % 4 != 0 || clear_floats < 0))
    return fail(HRT_ERR_INVALID_ARG, "x-pass: the buffer to clear must be 16-byte aligned, a multiple of 4 floats");
  CUtensorMap in_map, map_a, map_b;
  HRT_TRY(make_map<R1>(&in_map, in, static_cast<int>(n), 0));
  HRT_TRY(make_map<R1>(&map_a, a.out, static_cast<int>(n), a.n_out));
  if (TWO) HRT_TRY(make_map<R1>(&map_b, b.out, static_cast<int>(n), b.n_out));
  else map_b = map_a;
  const size_t smem = xpass_smem_bytes(n);
  int dev = 0, sms = 0;
  HRT_CUDA(cudaGetDevice(&dev));
  HRT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HRT_CUDA(cudaFuncSetAttribute(xpass_kernel<R1, TWO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem)));
  const int tiles = static_cast<int>(flat / G::TK);
  const int grid = std::min(tiles, sms);
  const double scale = -pref / (static_cast<double>(n) * n * n);
  const int64_t n4 = clear ? clear_floats / 4 : 0;
  xpass_kernel<R1, TWO><<<grid, kXThreads, smem, s>>>(in_map, map_a, map_b, nzc, tiles,
                                                      static_cast<float>(2.0 * M_PI / box), static_cast<float>(scale),
                                                      tw, a, b, err, n4 ? reinterpret_cast<float4*>(clear) : nullptr,
                                                      n4, (n4 + tiles - 1) / tiles);
  HRT_LAUNCHED("xpass_kernel");
  return HRT_OK;
}

hrt_status launch_xpass(const void* in, int64_t n, double box, double pref, const float2* tw, const XpassSet& a,
                        const XpassSet& b, int* err, cudaStream_t s, float* clear, int64_t clear_floats) {
  // every set has the x and y components (and z when n_out is 3): the x-pass stores V as d_y V [and d_z V]
  if (a.n_out < 2 || a.n_out > 3 || b.n_out == 1 || b.n_out < 0 || b.n_out > 3 || !err)
    return fail(HRT_ERR_INVALID_ARG, "x-pass: bad output sets");
  const bool two = b.n_out > 0;
  switch (n) {
    case 256:
      return two ? launch_r1<8, true>(in, n, box, pref, tw, a, b, err, clear, clear_floats, s)
                 : launch_r1<8, false>(in, n, box, pref, tw, a, b, err, clear, clear_floats, s);
    case 512:
      return two ? launch_r1<16, true>(in, n, box, pref, tw, a, b, err, clear, clear_floats, s)
                 : launch_r1<16, false>(in, n, box, pref, tw, a, b, err, clear, clear_floats, s);
    case 1024:
      return two ? launch_r1<32, true>(in, n, box, pref, tw, a, b, err, clear, clear_floats, s)
                 : launch_r1<32, false>(in, n, box, pref, tw, a, b, err, clear, clear_floats, s);
    default: return fail(HRT_ERR_INVALID_ARG, "x-pass needs a mesh side of 256, 512 or 1024");
  }
}

}  // namespace hrt
