// Shared-face form of the 3D patch sweep (combined colourised smoother,
// Algorithm 4, constant coefficient, degrees 3..8).  Included by patch_f64.cu
// and patch_f32.cu after patch_kernels.cuh and patch_launch.cuh (T = double
// or float).
//
// The local solver is exact, so the updated interior of patch j is
// A_j^{-1} (b_j - bar A_j bar u_j^0), bar u_j^0 its closure with the interior
// set to zero (App. A.3 with eqs. "main:4", "gather", "scatter").  The
// product bar A_j bar u_j^0 then involves only the closure boundary: its
// six faces.  With the two-cell 1D matrices M, K (interior rows, closure
// columns; M_I, K_I their interior columns) and the patch operator
// K (x) M (x) M + M (x) K (x) M + M (x) M (x) K (x fastest, axes x, y, z):
//   x face at closure x = f (all y, z; data v):
//     F1 = (M_y (x) M_z) v,  F2 = (K_y (x) M_z + M_y (x) K_z) v,
//     contribution K_x[:, f] (x) F1 + M_x[:, f] (x) F2;
//   y face at y = f (x interior, all z; data w):
//     G1 = (K_I,x (x) M_z + M_I,x (x) K_z) w,  G2 = (M_I,x (x) M_z) w,
//     contribution M_y[:, f] (x) G1 + K_y[:, f] (x) G2;
//   z face at z = f (x, y interior; data s):
//     H1 = (K_I,x (x) M_I,y + M_I,x (x) K_I,y) s,  H2 = (M_I,x (x) M_I,y) s,
//     contribution M_z[:, f] (x) H1 + K_z[:, f] (x) H2.
// F, G, H depend only on the face's node values and on its extent, and the
// face between two same-colour neighbours has the same extent in both
// patches: each face plane is evaluated once per colour (face kernel) and
// read by the two patches that share it (patch kernel).  Same-colour
// patches never write each other's closure, so the faces of a colour stay
// valid while its patches are updated.
#pragma once
#include "async.cuh"

namespace gmg {
namespace GMG_NS {

// Faces of one colour.  Patch (i_x, i_y, i_z) of the colour owns
//   x faces fx = i_x, i_x + 1 of X[(i_z c_y + i_y)(c_x + 1) + fx],
//   y faces fy = i_y, i_y + 1 of Y[(i_z (c_y + 1) + fy) c_x + i_x],
//   z faces fz = i_z, i_z + 1 of Z[(fz c_y + i_y) c_x + i_x].
// Each face holds two M x M fields: x faces F1, F2 as [l][j] (l the z row,
// j the y row), y faces G1, G2 as [l][i], z faces H1, H2 as [j][i]
// (i the x row), padded to a multiple of 16 bytes (face_fields elements);
// the families start at foff[0..2] elements.
struct FaceGeom {
  long long py, pz;
  int first[3], count[3];
  long long nf[3];
  long long foff[3];
};

__host__ __device__ constexpr int face_fields(int k) {
  return (2 * (2 * k - 1) * (2 * k - 1) + 16 / (int)sizeof(T) - 1) / (16 / (int)sizeof(T)) * (16 / (int)sizeof(T));
}

// acc + sum over the interior columns of row i of M_p (KIND 0) or K_p
// (KIND 1), x[a] the value at interior column a (closure column a + 1)
template <int K, int KIND>
__device__ __forceinline__ T patch_row_int(int i, const T (&x)[2 * K - 1], T acc = T(0)) {
  constexpr int C = 2 * K + 1, M = 2 * K - 1;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    if (a + 1 >= band_lo(i + 1, K) && a + 1 <= band_hi(i + 1, K)) {
      const T e = KIND == 0 ? c_Mp[off_patch(K) + i * C + a + 1] : c_Kp[off_patch(K) + i * C + a + 1];
      acc = fma(e, x[a], acc);
    }
  }
  return acc;
}

// element offset of the first node of face f of family fam (0 x, 1 y, 2 z):
// the face planes of patch (i_x, i_y, i_z) sit at its closure origin (index
// i) and at the next patch's (index i + 1); in-plane the data start at the
// closure origin (axes the face spans completely) or one node inside it
// (interior rows)
template <int K>
__device__ __forceinline__ long long face_origin(const FaceGeom& fg, int fam, long long f) {
  const int cx = fg.count[0], cy = fg.count[1];
  long long ix, iy, iz;
  if (fam == 0) {
    ix = f % (cx + 1);
    const long long r = f / (cx + 1);
    iy = r % cy;
    iz = r / cy;
  } else if (fam == 1) {
    ix = f % cx;
    const long long r = f / cx;
    iy = r % (cy + 1);
    iz = r / (cy + 1);
  } else {
    ix = f % cx;
    const long long r = f / cx;
    iy = r % cy;
    iz = r / cy;
  }
  const long long X = (fg.first[0] + 2 * ix - 1) * K + (fam == 0 ? 0 : 1);
  const long long Y = (fg.first[1] + 2 * iy - 1) * K + (fam == 2 ? 1 : 0);
  const long long Z = (fg.first[2] + 2 * iz - 1) * K;
  return X + fg.py * Y + fg.pz * Z;
}

// faces per CTA of the face kernel: enough first-stage lines for NT threads
template <int K, int NT>
struct FaceCfg {
  static constexpr int C = 2 * K + 1, M = 2 * K - 1;
  static constexpr int FX = NT / C > 0 ? NT / C : 1, FYZ = NT / M > 0 ? NT / M : 1;
  // per face: input, then the first-stage P and Q
  static constexpr int SX = C * C + 2 * C * M, SY = M * C + 2 * M * M, SZ = M * M + 2 * M * M;
  static constexpr int SMEM = cmax(FX * SX, cmax(FYZ * SY, FYZ * SZ)) * (int)sizeof(T);
};

// Face kernel: CTAs [0, bx) evaluate x faces, [bx, bx + by) y faces, the rest
// z faces, FX (FYZ) faces per CTA.  First stage: contract z (x and y faces,
// all closure rows of the two-cell matrices) or y (z faces, interior
// columns); second stage: contract the remaining in-plane axis.
template <int K, int NT>
__global__ void __launch_bounds__(NT) face_kernel(const T* __restrict__ u, T* __restrict__ faces,
                                                  const __grid_constant__ FaceGeom fg, int bx, int by) {
  using F = FaceCfg<K, NT>;
  constexpr int C = F::C, M = F::M, FS = face_fields(K);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* const S = reinterpret_cast<T*>(smem_raw);
  int fam, blk;
  if ((int)blockIdx.x < bx) { fam = 0; blk = blockIdx.x; }
  else if ((int)blockIdx.x < bx + by) { fam = 1; blk = blockIdx.x - bx; }
  else { fam = 2; blk = blockIdx.x - bx - by; }
  const int per = fam == 0 ? F::FX : F::FYZ;
  const long long f0 = (long long)blk * per;
  const int nq = (int)min((long long)per, fg.nf[fam] - f0);
  T* const out = faces + fg.foff[fam] + f0 * FS;
  if (fam == 0) {
    // ---- x faces: v[y][z] (C x C); P, Q[y][l] = (M_z, K_z) v[y][:] ----
    T* V = S;
    T* P = S + F::FX * C * C;
    T* Q = P + F::FX * C * M;
    for (int t = threadIdx.x; t < nq * C * C; t += NT) {
      const int q = t % nq, e = t / nq, y = e % C, z = e / C;  // faces fastest: nearby x planes
      V[q * C * C + y * C + z] = u[face_origin<K>(fg, 0, f0 + q) + fg.py * y + fg.pz * z];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq * C; t += NT) {
      const int q = t / C, y = t % C;
      T v[C];
#pragma unroll
      for (int z = 0; z < C; ++z) v[z] = V[q * C * C + y * C + z];
#pragma unroll
      for (int l = 0; l < M; ++l) {
        P[(q * C + y) * M + l] = patch_row<K, 0>(l, v);
        Q[(q * C + y) * M + l] = patch_row<K, 1>(l, v);
      }
    }
    __syncthreads();
    // F1[l][j] = (M_y P)[j][l], F2[l][j] = (K_y P + M_y Q)[j][l]
    for (int t = threadIdx.x; t < nq * M; t += NT) {
      const int q = t / M, l = t % M;
      T p[C], r[C];
#pragma unroll
      for (int y = 0; y < C; ++y) {
        p[y] = P[(q * C + y) * M + l];
        r[y] = Q[(q * C + y) * M + l];
      }
      T* o = out + (long long)q * FS + l * M;
#pragma unroll
      for (int j = 0; j < M; ++j) {
        o[j] = patch_row<K, 0>(j, p);
        o[M * M + j] = patch_row<K, 0>(j, r, patch_row<K, 1>(j, p));
      }
    }
    return;
  }
  T* P = S + F::FYZ * (fam == 1 ? M * C : M * M);
  T* Q = P + F::FYZ * M * M;
  if (fam == 1) {
    // ---- y faces: w[a][z] (a the interior x row); P, Q[a][l] = (M_z, K_z) w[a][:] ----
    T* W = S;
    for (int t = threadIdx.x; t < nq * M * C; t += NT) {
      const int a = t % M, e = t / M, z = e % C, q = e / C;  // x fastest: contiguous rows
      W[(q * M + a) * C + z] = u[face_origin<K>(fg, 1, f0 + q) + a + fg.pz * z];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq * M; t += NT) {
      const int q = t / M, a = t % M;
      T v[C];
#pragma unroll
      for (int z = 0; z < C; ++z) v[z] = W[(q * M + a) * C + z];
#pragma unroll
      for (int l = 0; l < M; ++l) {
        P[(q * M + a) * M + l] = patch_row<K, 0>(l, v);
        Q[(q * M + a) * M + l] = patch_row<K, 1>(l, v);
      }
    }
  } else {
    // ---- z faces: s[a][b] (interior x row a, y row b); P, Q[a][j] = (M_I, K_I) s[a][:] ----
    T* Sz = S;
    for (int t = threadIdx.x; t < nq * M * M; t += NT) {
      const int a = t % M, e = t / M, b = e % M, q = e / M;
      Sz[(q * M + a) * M + b] = u[face_origin<K>(fg, 2, f0 + q) + a + fg.py * b];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq * M; t += NT) {
      const int q = t / M, a = t % M;
      T v[M];
#pragma unroll
      for (int b = 0; b < M; ++b) v[b] = Sz[(q * M + a) * M + b];
#pragma unroll
      for (int j = 0; j < M; ++j) {
        P[(q * M + a) * M + j] = patch_row_int<K, 0>(j, v);
        Q[(q * M + a) * M + j] = patch_row_int<K, 1>(j, v);
      }
    }
  }
  __syncthreads();
  // y faces: G1[l][i] = (K_I P + M_I Q)[i][l], G2[l][i] = (M_I P)[i][l];
  // z faces: the same with l -> j (H1, H2)
  for (int t = threadIdx.x; t < nq * M; t += NT) {
    const int q = t / M, l = t % M;
    T p[M], r[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      p[a] = P[(q * M + a) * M + l];
      r[a] = Q[(q * M + a) * M + l];
    }
    T* o = out + (long long)q * FS + l * M;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      o[i] = patch_row_int<K, 0>(i, r, patch_row_int<K, 1>(i, p));
      o[M * M + i] = patch_row_int<K, 0>(i, p);
    }
  }
}

// The face kernel of FP64 problems in double-float arithmetic: the node
// values are read as doubles and split into float pairs, both stages
// accumulate in Dot2 form with the float-pair patch matrices, and the face
// fields are stored as float pairs (the same 8 bytes per entry as a double).
template <int K, int NT>
__global__ void __launch_bounds__(NT) face_kernel_df(const double* __restrict__ u, float2* __restrict__ faces,
                                                     const __grid_constant__ FaceGeom fg, int bx, int by) {
  using F = FaceCfg<K, NT>;
  constexpr int C = F::C, M = F::M, FS = face_fields(K);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* const S = reinterpret_cast<float2*>(smem_raw);
  int fam, blk;
  if ((int)blockIdx.x < bx) { fam = 0; blk = blockIdx.x; }
  else if ((int)blockIdx.x < bx + by) { fam = 1; blk = blockIdx.x - bx; }
  else { fam = 2; blk = blockIdx.x - bx - by; }
  const int per = fam == 0 ? F::FX : F::FYZ;
  const long long f0 = (long long)blk * per;
  const int nq = (int)min((long long)per, fg.nf[fam] - f0);
  float2* const out = faces + fg.foff[fam] + f0 * FS;
  auto ld = [](const float2 v) -> dfv { return {v.x, v.y}; };
  auto st = [](const dfv v) -> float2 { return make_float2(v.hi, v.lo); };
  if (fam == 0) {
    float2* V = S;
    float2* P = S + F::FX * C * C;
    float2* Q = P + F::FX * C * M;
    for (int t = threadIdx.x; t < nq * C * C; t += NT) {
      const int q = t % nq, e = t / nq, y = e % C, z = e / C;
      V[q * C * C + y * C + z] = st(df_from_double(u[face_origin<K>(fg, 0, f0 + q) + fg.py * y + fg.pz * z]));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq * C; t += NT) {
      const int q = t / C, y = t % C;
      dfv v[C];
#pragma unroll
      for (int z = 0; z < C; ++z) v[z] = ld(V[q * C * C + y * C + z]);
#pragma unroll
      for (int l = 0; l < M; ++l) {
        df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
        patch_row_df<K, 0>(l, v, a);
        patch_row_df<K, 1>(l, v, b);
        P[(q * C + y) * M + l] = st(df_acc_value(a));
        Q[(q * C + y) * M + l] = st(df_acc_value(b));
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq * M; t += NT) {
      const int q = t / M, l = t % M;
      dfv p[C], r[C];
#pragma unroll
      for (int y = 0; y < C; ++y) {
        p[y] = ld(P[(q * C + y) * M + l]);
        r[y] = ld(Q[(q * C + y) * M + l]);
      }
      float2* o = out + (long long)q * FS + l * M;
#pragma unroll
      for (int j = 0; j < M; ++j) {
        df_acc a = {0.f, 0.f}, b = {0.f, 0.f};
        patch_row_df<K, 0>(j, p, a);
        patch_row_df<K, 1>(j, p, b);
        patch_row_df<K, 0>(j, r, b);
        o[j] = st(df_acc_value(a));
        o[M * M + j] = st(df_acc_value(b));
      }
    }
    return;
  }
  float2* P = S + F::FYZ * (fam == 1 ? M * C : M * M);
  float2* Q = P + F::FYZ * M * M;
  if (fam == 1) {
    float2* W = S;
    for (int t = threadIdx.x; t < nq * M * C; t += NT) {
      const int a = t % M, e = t / M, z = e % C, q = e / C;
      W[(q * M + a) * C + z] = st(df_from_double(u[face_origin<K>(fg, 1, f0 + q) + a + fg.pz * z]));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq * M; t += NT) {
      const int q = t / M, a = t % M;
      dfv v[C];
#pragma unroll
      for (int z = 0; z < C; ++z) v[z] = ld(W[(q * M + a) * C + z]);
#pragma unroll
      for (int l = 0; l < M; ++l) {
        df_acc x = {0.f, 0.f}, y = {0.f, 0.f};
        patch_row_df<K, 0>(l, v, x);
        patch_row_df<K, 1>(l, v, y);
        P[(q * M + a) * M + l] = st(df_acc_value(x));
        Q[(q * M + a) * M + l] = st(df_acc_value(y));
      }
    }
  } else {
    float2* Sz = S;
    for (int t = threadIdx.x; t < nq * M * M; t += NT) {
      const int a = t % M, e = t / M, b = e % M, q = e / M;
      Sz[(q * M + a) * M + b] = st(df_from_double(u[face_origin<K>(fg, 2, f0 + q) + a + fg.py * b]));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq * M; t += NT) {
      const int q = t / M, a = t % M;
      dfv v[M];
#pragma unroll
      for (int b = 0; b < M; ++b) v[b] = ld(Sz[(q * M + a) * M + b]);
#pragma unroll
      for (int j = 0; j < M; ++j) {
        df_acc x = {0.f, 0.f}, y = {0.f, 0.f};
        patch_row_int_df<K, 0>(j, v, x);
        patch_row_int_df<K, 1>(j, v, y);
        P[(q * M + a) * M + j] = st(df_acc_value(x));
        Q[(q * M + a) * M + j] = st(df_acc_value(y));
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nq * M; t += NT) {
    const int q = t / M, l = t % M;
    dfv p[M], r[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      p[a] = ld(P[(q * M + a) * M + l]);
      r[a] = ld(Q[(q * M + a) * M + l]);
    }
    float2* o = out + (long long)q * FS + l * M;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      df_acc x = {0.f, 0.f}, y = {0.f, 0.f};
      patch_row_int_df<K, 1>(i, p, x);
      patch_row_int_df<K, 0>(i, r, x);
      patch_row_int_df<K, 0>(i, p, y);
      o[i] = st(df_acc_value(x));
      o[M * M + i] = st(df_acc_value(y));
    }
  }
}

// Shared-memory plan of the shared-face sweep, per patch (elements of T):
//   IN (NBUF copies): interior rows of b (TMA box rows of XB, as in the
//       closure kernel), then the face blocks X0 X1 Y0 Y1 Z0 Z1 of the patch
//       (two M x M fields each, padded to 16 bytes, copied by
//       cp.async.bulk); 128-byte multiple
//   WB: the FD work (M^3)
//   SUMS: Y0 + Y1 and Z0 + Z1 (two padded face blocks), the terms of the
//   centre rows
template <int K>
struct FaceSweepSmem {
  static constexpr int C = 2 * K + 1, M = 2 * K - 1;
  static constexpr int A = 16 / (int)sizeof(T);
  static constexpr int XB = (C + A - 1 + A - 1) / A * A;
  static constexpr int R128 = 128 / (int)sizeof(T);
  static constexpr int NBIN = (M * M * XB + R128 - 1) / R128 * R128;
  static constexpr int FS = face_fields(K);
  static constexpr int IN = (NBIN + 6 * FS + R128 - 1) / R128 * R128;
  static constexpr int WB = M * M * M;
  static constexpr int SUMS = 2 * FS;
  static constexpr int per_patch(int nbuf) { return nbuf * IN + WB + SUMS; }
  static constexpr int BOX_B = M * M * XB * (int)sizeof(T);
  static constexpr int FACE_BYTES = FS * (int)sizeof(T);
};

struct FaceSweepArgs {
  T* u;
  const T* faces;
  const T* dinv;
  int* err;
  long long py, pz;
  int first[3], count[3];
  int n_patches, ngroups;
  long long foff[3];
  double sb, omega;
};

// One colour of the sweep, shared-face form.  Persistent CTAs walk groups of
// PPC patches; lanes 0..PPC-1 of warp 0 issue, per patch, one TMA box of b
// and six bulk copies of its face blocks, all completing on the slot's
// mbarrier (bounded wait; an expired wait sets err and the kernel carries
// on).  With NBUF = 2 the next group streams in while the current one is
// computed.  Stages: r = sb b - (face contributions) per interior x line,
// forward FD x | forward FD y | forward FD z, times the FD diagonal,
// backward FD z (one z line per thread) | backward FD y | backward FD x +
// scatter
// u = omega d + (1 - omega) u_old.
template <int K, int NT, int PPC, int NBUF>
__global__ void __launch_bounds__(NT) patch_face_kernel(const __grid_constant__ FaceSweepArgs fa,
                                                        const __grid_constant__ CUtensorMap bmap) {
  using Z = FaceSweepSmem<K>;
  constexpr int C = Z::C, M = Z::M, XB = Z::XB, FS = Z::FS, LINES = M * M;
  // FP64: the FD transforms run in double-float arithmetic (pairs of floats
  // in WB; the diagonal's float pairs follow the FP64 diagonal in dinv)
  constexpr bool DF = sizeof(T) == 8;
  static_assert(PPC <= 32, "one lane of warp 0 issues the copies of one patch");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* const IN0 = reinterpret_cast<T*>(smem_raw + ((128 - (async::smem_u32(smem_raw) & 127)) & 127));
  T* const WB = IN0 + NBUF * PPC * Z::IN;
  float2* const WB2 = reinterpret_cast<float2*>(WB);  // used when DF: same element size
  const float2* const dinv_df = reinterpret_cast<const float2*>(fa.dinv + M * M * M);
  T* const SUMS = WB + PPC * Z::WB;
  __shared__ long long s_origin[2][PPC];
  __shared__ int s_x[2][PPC][3];     // closure origin (lattice coordinates)
  __shared__ long long s_face[2][PPC][6];  // element offsets of the six face blocks
  __shared__ int s_nvalid[2];
  __shared__ __align__(8) uint64_t s_bar[2];
  uint32_t phase = 0;
  bool wait_ok = true;
  const T om = (T)fa.omega, sb = (T)fa.sb;
  const int cx = fa.count[0], cy = fa.count[1];
  if (threadIdx.x == 0) {
    async::mbar_init(&s_bar[0], 1);
    async::mbar_init(&s_bar[1], 1);
  }
  __syncthreads();

  auto set_origins = [&](int grp, int slot) {
    const int nv = min(PPC, fa.n_patches - grp * PPC);
    if (threadIdx.x == 0) s_nvalid[slot] = nv;
    if (threadIdx.x < nv) {
      const int pid = grp * PPC + threadIdx.x;
      const int ix = pid % cx, rest = pid / cx, iy = rest % cy, iz = rest / cy;
      const int o0 = (fa.first[0] + 2 * ix - 1) * K, o1 = (fa.first[1] + 2 * iy - 1) * K,
                o2 = (fa.first[2] + 2 * iz - 1) * K;
      s_origin[slot][threadIdx.x] = o0 + fa.py * o1 + fa.pz * o2;
      s_x[slot][threadIdx.x][0] = o0;
      s_x[slot][threadIdx.x][1] = o1;
      s_x[slot][threadIdx.x][2] = o2;
      const long long fxi = ((long long)iz * cy + iy) * (cx + 1) + ix;
      const long long fyi = ((long long)iz * (cy + 1) + iy) * cx + ix;
      const long long fzi = ((long long)iz * cy + iy) * cx + ix;
      s_face[slot][threadIdx.x][0] = fa.foff[0] + fxi * FS;
      s_face[slot][threadIdx.x][1] = fa.foff[0] + (fxi + 1) * FS;
      s_face[slot][threadIdx.x][2] = fa.foff[1] + fyi * FS;
      s_face[slot][threadIdx.x][3] = fa.foff[1] + (fyi + cx) * FS;
      s_face[slot][threadIdx.x][4] = fa.foff[2] + fzi * FS;
      s_face[slot][threadIdx.x][5] = fa.foff[2] + (fzi + (long long)cy * cx) * FS;
    }
  };
  auto prefetch = [&](int slot) {
    if (threadIdx.x >= 32) return;
    const int nv = s_nvalid[slot];
    if (threadIdx.x == 0)
      async::mbar_arrive_expect_tx(&s_bar[slot], (uint32_t)(nv * (Z::BOX_B + 6 * Z::FACE_BYTES)));
    __syncwarp();
    const int q = threadIdx.x;
    if (q < nv) {
      T* dst = IN0 + (slot * PPC + q) * Z::IN;
      const int x0 = s_x[slot][q][0], xa = x0 - x0 % Z::A;
      async::tma_load_3d(dst, &bmap, xa, s_x[slot][q][1] + 1, s_x[slot][q][2] + 1, &s_bar[slot]);
#pragma unroll
      for (int f = 0; f < 6; ++f)
        async::bulk_load(dst + Z::NBIN + f * FS, fa.faces + s_face[slot][q][f], Z::FACE_BYTES, &s_bar[slot]);
    }
  };
  auto wait_gather = [&](int slot) {
    if (wait_ok && !async::mbar_wait(&s_bar[slot], (phase >> slot) & 1u)) wait_ok = false;
    phase ^= 1u << slot;
  };

  const int ngroups = fa.ngroups;
  int grp = blockIdx.x;
  if (NBUF == 2 && grp < ngroups) {
    set_origins(grp, 0);
    __syncthreads();
    prefetch(0);
  }
  for (int it = 0; grp < ngroups; grp += gridDim.x, ++it) {
    const int cur = NBUF == 2 ? (it & 1) : 0;
    if (NBUF == 1) {
      set_origins(grp, 0);
      __syncthreads();
      prefetch(0);
      wait_gather(0);
    } else if (grp + (int)gridDim.x < ngroups) {
      set_origins(grp + gridDim.x, cur ^ 1);
      __syncthreads();
      prefetch(cur ^ 1);
      wait_gather(cur);
    } else {
      wait_gather(cur);
    }
    __syncthreads();
    const int nvalid = s_nvalid[cur];
    const T* IN = IN0 + cur * PPC * Z::IN;

    // ---- centre rows: column 0 of the two-cell matrices is nonzero on rows
    // 0..K-1 and column 2K on rows K-1..M-1, and on row K-1 (the vertex row)
    // both equal the same cell-matrix entry, so a y (z) face term there is
    // that entry times the sum of the two faces' fields ----
    for (int idx = threadIdx.x; idx < nvalid * Z::SUMS; idx += NT) {
      const int q = idx / Z::SUMS, e = idx % Z::SUMS;
      const T* F = IN + q * Z::IN + Z::NBIN + (e < FS ? 2 * FS : 4 * FS) + e % FS;
      if constexpr (DF) {
        const float2* F2 = reinterpret_cast<const float2*>(F);
        const dfv v = df_add({F2[0].x, F2[0].y}, {F2[FS].x, F2[FS].y});
        reinterpret_cast<float2*>(SUMS)[idx] = make_float2(v.hi, v.lo);
      } else {
        SUMS[idx] = F[0] + F[FS];
      }
    }
    __syncthreads();

    // ---- r = sb b - face contributions on interior x line (j, l), then the
    // forward FD transform along x; result into WB ----
    for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {
      const int q = idx / LINES, ln = idx % LINES, j = ln % M, l = ln / M;
      const T* P = IN + q * Z::IN;
      const T* Bq = P + s_x[cur][q][0] % Z::A + 1 + (l * M + j) * XB;
      const T* FX = P + Z::NBIN;  // X0, X1: F1[l][j], F2[l][j]
      // the y-face fields row j needs (G1[l][.], G2[l][.]: Y0, Y1 or their
      // sum) and those of row l for the z faces (H1[j][.], H2[j][.])
      const T* FY = (j < K - 1 ? FX + 2 * FS : j > K - 1 ? FX + 3 * FS : SUMS + q * Z::SUMS) + l * M;
      const T* FZ = (l < K - 1 ? FX + 4 * FS : l > K - 1 ? FX + 5 * FS : SUMS + q * Z::SUMS + FS) + j * M;
      if constexpr (DF) {
        // the same residual in double-float: faces and sums are float pairs
        auto ld = [](const T* p, int i) -> dfv {
          const float2 v = reinterpret_cast<const float2*>(p)[i];
          return {v.x, v.y};
        };
        const dfv f10 = ld(FX, l * M + j), f20 = ld(FX, M * M + l * M + j);
        const dfv f11 = ld(FX, FS + l * M + j), f21 = ld(FX, FS + M * M + l * M + j);
        const int cj = j < K ? 0 : C - 1, cl = l < K ? 0 : C - 1;
        float myh, myl, kyh, kyl, mzh, mzl, kzh, kzl;
        patch_entry_df<K, 0, true>(j, cj, myh, myl);
        patch_entry_df<K, 1, true>(j, cj, kyh, kyl);
        patch_entry_df<K, 0, true>(l, cl, mzh, mzl);
        patch_entry_df<K, 1, true>(l, cl, kzh, kzl);
        const float sbf = (float)fa.sb;  // h^{2-d} = n, exact in float
        dfv rd[M], yd[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const dfv bb = df_mul(df_from_double(Bq[i]), {sbf, 0.f});
          df_acc acc = {bb.hi, bb.lo};
          float h, lo;
          if (band_lo(i + 1, K) == 0) {
            patch_entry_df<K, 1, true>(i, 0, h, lo);
            df_acc_add(acc, h, lo, f10);
            patch_entry_df<K, 0, true>(i, 0, h, lo);
            df_acc_add(acc, h, lo, f20);
          }
          if (band_hi(i + 1, K) == 2 * K) {
            patch_entry_df<K, 1, true>(i, C - 1, h, lo);
            df_acc_add(acc, h, lo, f11);
            patch_entry_df<K, 0, true>(i, C - 1, h, lo);
            df_acc_add(acc, h, lo, f21);
          }
          df_acc_add(acc, kyh, kyl, ld(FY, M * M + i));
          df_acc_add(acc, myh, myl, ld(FY, i));
          df_acc_add(acc, kzh, kzl, ld(FZ, M * M + i));
          df_acc_add(acc, mzh, mzl, ld(FZ, i));
          rd[i] = df_acc_value(acc);
        }
        fd_forward_df<K>(rd, yd);
        float2* R = WB2 + q * Z::WB + M * ln;
#pragma unroll
        for (int i = 0; i < M; ++i) R[i] = make_float2(yd[i].hi, yd[i].lo);
        continue;
      }
      const T f10 = FX[l * M + j], f20 = FX[M * M + l * M + j];
      const T f11 = FX[FS + l * M + j], f21 = FX[FS + M * M + l * M + j];
      // column 0 (rows up to K-1) or 2K of rows j and l
      const int oj = off_patch(K) + j * C + (j < K ? 0 : C - 1);
      const int ol = off_patch(K) + l * C + (l < K ? 0 : C - 1);
      const T my = c_Mp[oj], ky = c_Kp[oj], mz = c_Mp[ol], kz = c_Kp[ol];
      T r[M], y[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        T acc = sb * Bq[i];
        if (band_lo(i + 1, K) == 0)
          acc = fma(-c_Kp[off_patch(K) + i * C], f10, fma(-c_Mp[off_patch(K) + i * C], f20, acc));
        if (band_hi(i + 1, K) == 2 * K)
          acc = fma(-c_Kp[off_patch(K) + i * C + C - 1], f11, fma(-c_Mp[off_patch(K) + i * C + C - 1], f21, acc));
        acc = fma(-my, FY[i], fma(-ky, FY[M * M + i], acc));
        r[i] = fma(-mz, FZ[i], fma(-kz, FZ[M * M + i], acc));
      }
      fd_forward<K>(r, y);
      T* R = WB + q * Z::WB + M * ln;
#pragma unroll
      for (int i = 0; i < M; ++i) R[i] = y[i];
    }
    __syncthreads();
    // ---- local solve by fast diagonalisation (App. A.3), in place in WB ----
    for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {  // forward y
      const int q = idx / LINES, l = idx % LINES;
      if constexpr (DF) fd_smem_line_df<K, true>(WB2 + q * Z::WB + (l % M) + (l / M) * M * M, M);
      else fd_smem_line<K, true>(WB + q * Z::WB + (l % M) + (l / M) * M * M, M);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {  // forward z, diagonal, backward z
      const int q = idx / LINES, l = idx % LINES;
      if constexpr (DF) fd_smem_line_solve_df<K>(WB2 + q * Z::WB + l, M * M, dinv_df + l, M * M);
      else fd_smem_line_solve<K>(WB + q * Z::WB + l, M * M, fa.dinv + l, M * M);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {  // backward y
      const int q = idx / LINES, l = idx % LINES;
      if constexpr (DF) fd_smem_line_df<K, false>(WB2 + q * Z::WB + (l % M) + (l / M) * M * M, M);
      else fd_smem_line<K, false>(WB + q * Z::WB + (l % M) + (l / M) * M * M, M);
    }
    __syncthreads();
    // ---- backward FD along x and scatter (eq. "scatter") ----
    for (int idx = threadIdx.x; idx < nvalid * LINES; idx += NT) {
      const int q = idx / LINES, l = idx % LINES;
      T d[M];
      if constexpr (DF) {
        const float2* R = WB2 + q * Z::WB + M * l;
        dfv yv[M], dd[M];
#pragma unroll
        for (int i = 0; i < M; ++i) yv[i] = {R[i].x, R[i].y};
        fd_backward_df<K>(yv, dd);
#pragma unroll
        for (int i = 0; i < M; ++i) d[i] = df_to_double(dd[i]);
      } else {
        const T* R = WB + q * Z::WB + M * l;
        T yv[M];
#pragma unroll
        for (int i = 0; i < M; ++i) yv[i] = R[i];
        fd_backward<K>(yv, d);
      }
      T* __restrict__ row = fa.u + s_origin[cur][q] + 1 + fa.py * (l % M + 1) + fa.pz * (l / M + 1);
      if (om == T(1)) {
#pragma unroll
        for (int i = 0; i < M; ++i) row[i] = d[i];
      } else {
#pragma unroll
        for (int i = 0; i < M; ++i) row[i] = fma(om, d[i], (T(1) - om) * row[i]);
      }
    }
    async::fence_proxy_async();  // reads of the buffers before the next copies write them
    __syncthreads();
  }
  if (!wait_ok) atomicExch(fa.err, GMG_ERR_TIMEOUT);
}

// ---- host side ----

// patches per CTA, threads and input buffers of the shared-face sweep
template <int K>
struct FaceSweepCfg {
  // FP64 (double-float arithmetic, bound by FP32 issue) at k = 3, 4: one input
  // buffer, which leaves room for more resident CTAs (measured on GB300 at
  // 64^3: k = 3 1.30 -> 1.12 ms, k = 4 3.16 -> 3.03 ms per sweep); FP32 and
  // the other degrees keep the double-buffered inputs
  static constexpr bool F64 = sizeof(T) == 8;
  static constexpr int PPC = K == 3 ? (F64 ? 5 : 10) : K == 4 ? 5 : K == 5 ? 3 : K == 6 ? 2 : 1;
  // (FP32 k = 7: 160 threads, 2.75 -> 2.67 ms per 48^3 sweep)
  static constexpr int NT = K == 7 ? (F64 ? 192 : 160) : K == 3 && F64 ? 128 : 256;
  static constexpr int NBUF = (K <= 4 && !F64) || K == 7 ? 2 : 1;
  static constexpr int SMEM = PPC * FaceSweepSmem<K>::per_patch(NBUF) * (int)sizeof(T) + 128;
  static_assert(SMEM <= 227 * 1024, "shared-face sweep exceeds the shared memory of a CTA");
  static_assert(PPC * (2 * K - 1) * (2 * K - 1) <= NT + 32 * 2,
                "the interior lines of a patch group should take about one pass of the CTA's threads");
};
constexpr int kFaceThreads = 128;

static FaceGeom face_geom(const PatchLaunch& pl) {
  FaceGeom fg;
  fg.py = pl.g.py;
  fg.pz = pl.g.pz;
  for (int a = 0; a < 3; ++a) {
    fg.first[a] = pl.first[a];
    fg.count[a] = pl.count[a];
  }
  const long long cx = pl.count[0], cy = pl.count[1], cz = pl.count[2];
  fg.nf[0] = (cx + 1) * cy * cz;
  fg.nf[1] = cx * (cy + 1) * cz;
  fg.nf[2] = cx * cy * (cz + 1);
  const long long fs = face_fields(pl.g.k);
  fg.foff[0] = 0;
  fg.foff[1] = fg.nf[0] * fs;
  fg.foff[2] = fg.foff[1] + fg.nf[1] * fs;
  return fg;
}

template <int K>
static int face_sweep_impl(const PatchLaunch& pl, T* u, const T* b, const T* dinv, T* faces, cudaStream_t s) {
  using FC = FaceCfg<K, kFaceThreads>;
  using SC = FaceSweepCfg<K>;
  using Z = FaceSweepSmem<K>;
  // FP64 problems evaluate the faces in double-float (float-pair fields)
  auto fk = [] {
    if constexpr (sizeof(T) == 8) return face_kernel_df<K, kFaceThreads>;
    else return face_kernel<K, kFaceThreads>;
  }();
  auto pk = patch_face_kernel<K, SC::NT, SC::PPC, SC::NBUF>;
  static PerDevice<int> per_sm_dev;
  int* const per_sm_p = per_sm_dev.get();
  if (!per_sm_p) return GMG_ERR_CUDA;
  int& per_sm = *per_sm_p;
  if (per_sm == 0) {
    if (prepare(fk, FC::SMEM) != GMG_OK || prepare(pk, SC::SMEM) != GMG_OK) return GMG_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pk, SC::NT, SC::SMEM) != cudaSuccess ||
        per_sm <= 0)
      return GMG_ERR_CUDA;
  }
  const FaceGeom fg = face_geom(pl);
  const long long bx = (fg.nf[0] + FC::FX - 1) / FC::FX, by = (fg.nf[1] + FC::FYZ - 1) / FC::FYZ,
                  bz = (fg.nf[2] + FC::FYZ - 1) / FC::FYZ;
  if (bx + by + bz > (1LL << 31) - 1) return GMG_ERR_UNSUPPORTED;
  if constexpr (sizeof(T) == 8)
    fk<<<(unsigned)(bx + by + bz), kFaceThreads, FC::SMEM, s>>>(u, reinterpret_cast<float2*>(faces), fg, (int)bx,
                                                                (int)by);
  else
    fk<<<(unsigned)(bx + by + bz), kFaceThreads, FC::SMEM, s>>>(u, faces, fg, (int)bx, (int)by);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return GMG_ERR_CUDA;

  FaceSweepArgs fa;
  fa.u = u;
  fa.faces = faces;
  fa.dinv = dinv;
  fa.err = device_wait_flag();
  if (!fa.err) return GMG_ERR_CUDA;
  fa.py = pl.g.py;
  fa.pz = pl.g.pz;
  for (int a = 0; a < 3; ++a) {
    fa.first[a] = pl.first[a];
    fa.count[a] = pl.count[a];
    fa.foff[a] = fg.foff[a];
  }
  fa.n_patches = pl.n_patches;
  fa.ngroups = (pl.n_patches + SC::PPC - 1) / SC::PPC;
  fa.sb = pl.sb;
  fa.omega = pl.omega;
  CUtensorMap bmap;
  if (!tma_encode(&bmap, b, (int)sizeof(T), 3, pl.g.N, pl.g.py, pl.g.pz, Z::XB, Z::M)) return GMG_ERR_CUDA;
  const int grid = std::min(fa.ngroups, per_sm * sm_count());
  pk<<<grid, SC::NT, SC::SMEM, s>>>(fa, bmap);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GMG_OK : GMG_ERR_CUDA;
}

// elements of the face buffer for one colour launch of pl's geometry
inline long long face_buffer_elems_t(const PatchLaunch& pl) {
  const FaceGeom fg = face_geom(pl);
  return (fg.nf[0] + fg.nf[1] + fg.nf[2]) * face_fields(pl.g.k);
}

}  // namespace GMG_NS
}  // namespace gmg

namespace gmg {

template <>
int launch_patch_faces<GMG_T>(const PatchLaunch& pl, GMG_T* u, const GMG_T* b, const GMG_T* dinv, GMG_T* faces,
                              cudaStream_t s) {
  if (pl.g.dim != 3 || pl.g.k < 3 || pl.g.k > 8 || pl.mode != 0 || pl.plist || !faces)
    return GMG_ERR_UNSUPPORTED;
  if (!tma_vector_ok(b, (int)sizeof(GMG_T), 3, pl.g.py, pl.g.pz)) return GMG_ERR_UNSUPPORTED;
  if (pl.n_patches <= 0) return GMG_OK;
  switch (pl.g.k) {
    case 3: return GMG_NS::face_sweep_impl<3>(pl, u, b, dinv, faces, s);
    case 4: return GMG_NS::face_sweep_impl<4>(pl, u, b, dinv, faces, s);
    case 5: return GMG_NS::face_sweep_impl<5>(pl, u, b, dinv, faces, s);
    case 6: return GMG_NS::face_sweep_impl<6>(pl, u, b, dinv, faces, s);
    case 7: return GMG_NS::face_sweep_impl<7>(pl, u, b, dinv, faces, s);
    default: return GMG_NS::face_sweep_impl<8>(pl, u, b, dinv, faces, s);
  }
}

template <>
long long face_buffer_elems<GMG_T>(const PatchLaunch& pl) {
  return GMG_NS::face_buffer_elems_t(pl);
}

}  // namespace gmg
