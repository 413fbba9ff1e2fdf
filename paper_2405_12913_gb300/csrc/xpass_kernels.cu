// The x-pass of the split Poisson solve: with the density transformed over (y, z) by batched 2D cuFFT plans, one
// kernel does, per pencil (ky, kz) along x, the forward x-FFT, the fused k-space step (Green's function of the
// Poisson equation of Sec. 2, derivative i k_j, per-axis deconvolution and smoothing, learned factor g) and the
// inverse x-FFTs of the gradient spectra; batched 2D C2R plans finish the gradient fields.  Together with the 2D
// plans this reads and writes every spectrum once less than a 3D R2C, a separate k-space kernel and 3D C2Rs.
//
// FFT along x (n = 32 R1 points): four-step, x = l + 32 m, k = k1 + R1 k2.  A warp holds 32 complex values per
// lane: lane l first holds x = l + 32 m of its P = 32 / R1 pencils, does the R1-point DFTs over m in registers,
// applies the twiddles W_n^(l k1), transposes through its pencils' columns of the shared tile, and does the
// 32-point DFT over l in registers, so that lane (p, k1) holds X[k1 + R1 k2] for all k2.  The inverse runs the
// same steps backwards and returns to the first layout.  The gradient spectra are linear in the pencil: for a
// pencil (ky, kz) the y and z components are d_y V and d_z V with V = IFFT_x(i c X), so a filter set needs two
// inverse transforms (V and the x component) for its three outputs.
//
// Tiles: a CTA of 8 warps owns the pencils (ky, kz0 .. kz0 + 8P - 1) for all x: rows of 8P contiguous complex
// values in the [x][ky][kz] half spectra (the last tile holds only the Nyquist column kz = n/2).  Persistent CTAs; the next tile is copied into the second shared buffer with cp.async while
// the current one is transformed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "common.h"
#include "xpass.h"

namespace hrt {

namespace {

constexpr int kXWarps = 8;

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

// Slot of the transposed element (k1, l) in a pencil's column: the XOR keeps both the row-wise writes and the
// column-wise reads of a warp on distinct bank pairs (the column stride LD is odd).
__device__ __forceinline__ int slot(int k1, int l) { return k1 * 32 + (l ^ k1); }

__device__ __forceinline__ void cp_async8(float2* dst, const float2* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ float learned_factor(const XpassSet& s, float kmag) {
  if (s.g == nullptr) return 1.f;
  const float t = kmag * s.g_inv_dk;
  if (t >= static_cast<float>(s.g_nk - 1)) return 1.f;
  const int i = static_cast<int>(t);
  const float w = t - static_cast<float>(i);
  return __ldg(s.g + i) * (1.f - w) + __ldg(s.g + i + 1) * w;
}

struct TileGeom {
  int ky, kz0, width;
};

__device__ __forceinline__ TileGeom tile_geom(int tile, int kz_tiles, int tk, int nzc) {
  TileGeom t;
  t.ky = tile / kz_tiles;
  t.kz0 = (tile - t.ky * kz_tiles) * tk;
  t.width = min(tk, nzc - t.kz0);
  return t;
}

// Copies the tile's valid columns of all n rows into shared memory (8-byte cp.async, TK threads per row).
template <int TK, int LD>
__device__ __forceinline__ void load_tile(const float2* __restrict__ in, int n, int nzp, const TileGeom& g,
                                          float2* dst) {
  for (int e = threadIdx.x; e < n * TK; e += blockDim.x) {
    const int x = e / TK, c = e - x * TK;
    if (c < g.width) cp_async8(dst + x * LD + c, in + (static_cast<int64_t>(x) * n + g.ky) * nzp + g.kz0 + c);
  }
}

template <int TK, int LD>
__device__ __forceinline__ void store_tile(float2* __restrict__ out, int n, int nzp, const TileGeom& g,
                                           const float2* src) {
  for (int e = threadIdx.x; e < n * TK; e += blockDim.x) {
    const int x = e / TK, c = e - x * TK;
    if (c < g.width) out[(static_cast<int64_t>(x) * n + g.ky) * nzp + g.kz0 + c] = src[x * LD + c];
  }
}

// Inverse x-FFT from layout B (lane (p, k1), u[k2] = X[k1 + R1 k2]) to layout A (lane l, u[p R1 + n2] =
// x[l + 32 n2]) through the warp's columns col0 .. col0 + P - 1 of the tile.
template <int R1>
__device__ __forceinline__ void inverse_x(float2 (&u)[32], float2* T, int col0, const float2* twi, int lane) {
  constexpr int P = 32 / R1, LD = kXWarps * P + 1;
  dft<32, true, 0>(u);
#pragma unroll
  for (int n1 = 1; n1 < 32; ++n1) u[n1] = cmul(u[n1], twi[n1 * 32 + lane]);
  const int pp = lane / R1, k1 = lane - pp * R1;
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) T[slot(k1, n1) * LD + col0 + pp] = u[n1];
  __syncwarp();
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int j = 0; j < R1; ++j) u[p * R1 + j] = T[slot(j, lane) * LD + col0 + p];
  __syncwarp();
  DftPencils<R1, true, P>::run(u);
}

// c(k) = Green's function x per-axis filter factors x learned g at kx = k1 + R1 k2 (the k-space kernel's factor).
template <int R1>
__device__ __forceinline__ float filter_c(const XpassSet& s, const float* wx, int n, int k1, int k2, float kf,
                                          float scale, float k2yz, float cyz) {
  const int kx = k1 + R1 * k2;
  const int nx = kx < (n >> 1) ? kx : kx - n;
  const float kxf = kf * nx;
  const float kk = kxf * kxf + k2yz;
  const float green = kk > 0.f ? __fdividef(scale, kk) : 0.f;
  float c = green * wx[kx] * cyz;
  if (s.g != nullptr) c *= learned_factor(s, sqrtf(kk));
  return c;
}

__device__ __forceinline__ float dx_of(int kx, int n, float kf) {
  const int nx = kx < (n >> 1) ? kx : kx - n;
  return nx == -(n >> 1) ? 0.f : kf * nx;
}

// u[k2] = d(kx) Y[k2] at kx = k1 + R1 k2, with Y = i c X: computed here from X (PRE false) or given in X
// (PRE true); d = d_x of each kx when with_dx, else 1.
template <int R1, bool PRE>
__device__ __forceinline__ void filtered(const float2 (&X)[32], float2 (&u)[32], const XpassSet& s,
                                         const float* wx, int n, int k1, float kf, float scale, float k2yz,
                                         float cyz, bool with_dx) {
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) {
    const float d = with_dx ? dx_of(k1 + R1 * k2, n, kf) : 1.f;
    if (PRE) {
      u[k2] = make_float2(d * X[k2].x, d * X[k2].y);
    } else {
      const float c = d * filter_c<R1>(s, wx, n, k1, k2, kf, scale, k2yz, cyz);
      u[k2] = make_float2(-c * X[k2].y, c * X[k2].x);
    }
  }
}

// The gradient spectra of one filter set for the tile: the x component, then V = IFFT_x(i c X), stored once
// scaled by d_y and once by d_z; each transform's result is written to the tile's rows and stored by the CTA.
template <int R1, bool PRE>
__device__ __forceinline__ void one_set(const XpassSet& s, const float* wx, const float2 (&X)[32], float2* T,
                                        const TileGeom& g, int col0, int k1, int lane, bool busy, int n, int nzp,
                                        float kf, float scale, int kz, float k2yz, float dy, int64_t plane,
                                        const float2* twi) {
  constexpr int P = 32 / R1, TK = kXWarps * P, LD = TK + 1;
  const int half = n >> 1;
  const float cyz = __ldg(s.wxy + g.ky) * __ldg(s.wz + kz);
  float2 u[32];
  if (busy) {
    filtered<R1, PRE>(X, u, s, wx, n, k1, kf, scale, k2yz, cyz, true);
    inverse_x<R1>(u, T, col0, twi, lane);
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int j = 0; j < R1; ++j) T[(lane + 32 * j) * LD + col0 + p] = u[p * R1 + j];
  }
  __syncthreads();
  store_tile<TK, LD>(s.out, n, nzp, g, T);
  __syncthreads();
  if (busy) {
    filtered<R1, PRE>(X, u, s, wx, n, k1, kf, scale, k2yz, cyz, false);
    inverse_x<R1>(u, T, col0, twi, lane);
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int j = 0; j < R1; ++j) T[(lane + 32 * j) * LD + col0 + p] = u[p * R1 + j];
  }
  __syncthreads();
  // y and z components in one pass over V: d_y is the tile's, d_z each column's
  float2* out_y = s.out + plane;
  float2* out_z = s.n_out > 2 ? s.out + 2 * plane : nullptr;
  for (int e = threadIdx.x; e < n * TK; e += blockDim.x) {
    const int x = e / TK, c = e - x * TK;
    if (c >= g.width) continue;
    const float2 v = T[x * LD + c];
    const int64_t o = (static_cast<int64_t>(x) * n + g.ky) * nzp + g.kz0 + c;
    out_y[o] = make_float2(dy * v.x, dy * v.y);
    if (out_z) {
      const int kzc = g.kz0 + c;
      const float dz = kzc == half ? 0.f : kf * kzc;
      out_z[o] = make_float2(dz * v.x, dz * v.y);
    }
  }
  __syncthreads();
}

template <int R1, bool TWO>
__global__ void __launch_bounds__(kXWarps * 32, 1)
    xpass_kernel(const float2* __restrict__ in, int n, int nzc, int nzp, int kz_tiles, float kf, float scale,
                 const float2* __restrict__ tw, XpassSet a, XpassSet b) {
  constexpr int P = 32 / R1, TK = kXWarps * P, LD = TK + 1;
  extern __shared__ float2 sm[];
  float2* twf = sm;             // [R1][32]: W_n^(l k1)
  float2* twi = twf + R1 * 32;  // [32][32]: W_n^(-n1 k1(lane))
  float* wxa = reinterpret_cast<float*>(twi + 32 * 32);
  float* wxb = wxa + n;
  float2* const buf0 = reinterpret_cast<float2*>(wxb + n);
  float2* const buf1 = buf0 + n * LD;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < R1 * 32 + 32 * 32; i += blockDim.x) sm[i] = tw[i];
  for (int i = tid; i < n; i += blockDim.x) {
    wxa[i] = __ldg(a.wxy + i);
    wxb[i] = TWO ? __ldg(b.wxy + i) : 0.f;
  }
  const int n_tiles = n * kz_tiles;
  const int64_t plane = static_cast<int64_t>(n) * n * nzp;
  const int half = n >> 1;
  const int col0 = warp * P;
  const int pp = lane / R1, k1 = lane - pp * R1;
  int cur = 0;
  if (static_cast<int>(blockIdx.x) < n_tiles)
    load_tile<TK, LD>(in, n, nzp, tile_geom(blockIdx.x, kz_tiles, TK, nzc), buf0);
  cp_async_commit();
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    if (next < n_tiles) load_tile<TK, LD>(in, n, nzp, tile_geom(next, kz_tiles, TK, nzc), cur ? buf0 : buf1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const TileGeom g = tile_geom(tile, kz_tiles, TK, nzc);
    float2* T = cur ? buf1 : buf0;
    const bool busy = col0 < g.width;
    // ---- forward x-FFT of the warp's pencils: X[k2] = spectrum at kx = k1 + R1 k2 of pencil col0 + pp
    float2 X[32];
    if (busy) {
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int m = 0; m < R1; ++m) X[p * R1 + m] = T[(lane + 32 * m) * LD + col0 + p];
      __syncwarp();
      DftPencils<R1, false, P>::run(X);
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int j = 1; j < R1; ++j) X[p * R1 + j] = cmul(X[p * R1 + j], twf[j * 32 + lane]);
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int j = 0; j < R1; ++j) T[slot(j, lane) * LD + col0 + p] = X[p * R1 + j];
      __syncwarp();
#pragma unroll
      for (int l = 0; l < 32; ++l) X[l] = T[slot(k1, l) * LD + col0 + pp];
      __syncwarp();
      dft<32, false, 0>(X);
    }
    // pencil frequencies (ky, kz); columns past the tile's width hold no pencil and are not stored
    const int kz = min(g.kz0 + col0 + pp, half);
    const int ny = g.ky < half ? g.ky : g.ky - n;
    const float kyf = kf * ny, kzf = kf * kz;
    const float k2yz = kyf * kyf + kzf * kzf;
    const float dy = ny == -half ? 0.f : kyf;
    if (TWO) {
      one_set<R1, false>(a, wxa, X, T, g, col0, k1, lane, busy, n, nzp, kf, scale, kz, k2yz, dy, plane, twi);
      one_set<R1, false>(b, wxb, X, T, g, col0, k1, lane, busy, n, nzp, kf, scale, kz, k2yz, dy, plane, twi);
    } else {
      // one filter set: Y = i c X once, in place
      if (busy) {
        const float cyz = __ldg(a.wxy + g.ky) * __ldg(a.wz + kz);
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const float c = filter_c<R1>(a, wxa, n, k1, k2, kf, scale, k2yz, cyz);
          X[k2] = make_float2(-c * X[k2].y, c * X[k2].x);
        }
      }
      one_set<R1, true>(a, wxa, X, T, g, col0, k1, lane, busy, n, nzp, kf, scale, kz, k2yz, dy, plane, twi);
    }
    cur ^= 1;
  }
  cp_async_wait<0>();
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

template <int R1, bool TWO>
static hrt_status launch_r1(const void* in, int64_t n, double box, double pref, const float2* tw,
                            const XpassSet& a, const XpassSet& b, cudaStream_t s) {
  constexpr int P = 32 / R1, LD = kXWarps * P + 1;
  const int nzc = static_cast<int>(n / 2 + 1), nzp = static_cast<int>(xpass_row(n));
  const int kz_tiles = static_cast<int>((n / 2) / (kXWarps * P) + 1);
  const size_t smem = (static_cast<size_t>(R1) * 32 + 32 * 32) * sizeof(float2) + 2 * n * sizeof(float) +
                      2 * static_cast<size_t>(n) * LD * sizeof(float2);
  int dev = 0, sms = 0;
  HRT_CUDA(cudaGetDevice(&dev));
  HRT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HRT_CUDA(cudaFuncSetAttribute(xpass_kernel<R1, TWO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem)));
  const int tiles = static_cast<int>(n) * kz_tiles;
  const int grid = std::min(tiles, sms);
  const double scale = -pref / (static_cast<double>(n) * n * n);
  xpass_kernel<R1, TWO><<<grid, kXWarps * 32, smem, s>>>(static_cast<const float2*>(in), static_cast<int>(n), nzc, nzp,
                                                    kz_tiles, static_cast<float>(2.0 * M_PI / box),
                                                    static_cast<float>(scale), tw, a, b);
  HRT_LAUNCHED("xpass_kernel");
  return HRT_OK;
}

hrt_status launch_xpass(const void* in, int64_t n, double box, double pref, const float2* tw, const XpassSet& a,
                        const XpassSet& b, cudaStream_t s) {
  const bool two = b.n_out > 0;
  switch (n) {
    case 256: return two ? launch_r1<8, true>(in, n, box, pref, tw, a, b, s) : launch_r1<8, false>(in, n, box, pref, tw, a, b, s);
    case 512: return two ? launch_r1<16, true>(in, n, box, pref, tw, a, b, s) : launch_r1<16, false>(in, n, box, pref, tw, a, b, s);
    case 1024: return two ? launch_r1<32, true>(in, n, box, pref, tw, a, b, s) : launch_r1<32, false>(in, n, box, pref, tw, a, b, s);
    default: return fail(HRT_ERR_INVALID_ARG, "x-pass needs a mesh side of 256, 512 or 1024");
  }
}

}  // namespace hrt
