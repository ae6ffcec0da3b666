// Octree-AMR ray casting: the batch kernel's device code, for sm_103a.
//
// One thread traces one pixel's ray (Sec. 2.2 casts a single ray per pixel).
// Warps take 2-D pixel tiles from a device work queue shared by every camera of
// a batch (Sec. 3.2 hands work to whichever worker is free), so cameras of
// uneven size keep every SM busy until the last tile.
//
// Per ray:
//   set-up  : pixel centre in IEEE double (the only FP64 step of the FP32
//             kernels) from the camera's per-column and per-row offsets,
//             rounded to the 2^-36 lattice; box entry by exact comparisons of
//             rational crossing times.
//   descent : from the root down to the leaf holding the ray (Sec. 2.2),
//             choosing children by the exact side of the mid-planes at the
//             entry time; stops at a leaf or at the camera's level (Sec. 2).
//   step    : three 32-bit terms give the exact order of the cell's exit
//             times on the three axes; the chord is an exact integer time
//             difference times per-camera factors; value x chord is added;
//             the next cell is the same oct's neighbour (a bit flip of the
//             cell index) or the oct named by a face link (a coarser leaf, or
//             the end of the box); refined neighbours are descended into.
//             Per-camera tables indexed by the (entry, exit) axes and by the
//             set of stepped axes replace per-axis selects on this path.
//             Without links (the no-allocation entry point) the neighbour is
//             reached through the stack of ancestor octs instead.
//
// Oct records are 8 bytes {index of the first child oct, 8-bit refinement
// mask | level << 8}; siblings are contiguous, so the child of cell c is
// first + popc(mask & ((1 << c) - 1)).  Each oct also has a 64-byte link block:
// six 8-byte face links {neighbour, the neighbour oct's mask | level << 8} and
// the oct's packed corner coordinates.  Field values are one array per field,
// indexed oct * 8 + cell.
//
// Included by amr_kernels.cu (the kernels at the default register cap and
// the launch functions) and amr_kernels_caps.cu (the other caps), which
// compile in parallel.
#pragma once

#include "amr_internal.h"
#include "amr.h"

namespace amr {
namespace {

constexpr long long kBox = 1LL << kFixBits;
constexpr int kStepCap = 1 << 25;  // no ray at level <= 22 visits this many leaves

template <typename T>
__device__ __forceinline__ T sel3(int i, T a, T b, T c) { return i == 0 ? a : (i == 1 ? b : c); }

// (density, v_x, v_y, v_z) of one cell from the packed array: one 16-byte
// load for float fields, two for double.
template <typename F>
struct Pack4 {
  F x, y, z, w;
};
template <typename F>
__device__ __forceinline__ Pack4<F> load_pack(const void* base, uint32_t cell) {
  if constexpr (sizeof(F) == 8) {
    const double2* p = static_cast<const double2*>(base) + 2 * (size_t)cell;
    const double2 a = __ldg(p), b = __ldg(p + 1);
    return {a.x, a.y, b.x, b.y};
  } else {
    const float4 a = __ldg(static_cast<const float4*>(base) + cell);
    return {a.x, a.y, a.z, a.w};
  }
}

template <typename F>
__device__ __forceinline__ F load_field(const void* base, size_t idx) {
  return __ldg(static_cast<const F*>(base) + idx);
}

// Compensated float sums.  Written with explicit round-to-nearest intrinsics so
// no step is contracted or reassociated.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

__device__ __forceinline__ void neumaier_add(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float e = fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
  c = __fadd_rn(c, e);
  s = t;
}

// A ray's accumulators: FP64 sums (s = column / denominator, n = weighted
// numerator, m = maximum), or FP32 ones with their compensation terms.
struct RayOut {
  double s, n, m;
  float sf, cs, nf, cn, mf;
  int count;
};

template <int PREC, int MODE, bool NB, typename F, bool PACKED = false>
__device__ __forceinline__ RayOut trace_ray(const BatchArgs& A, const CamDev& cam, int i, int j) {
  RayOut res{0.0, 0.0, 0.0, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0};

  // ---- ray set-up: FP64 pixel centre, quantised origin ----------------------
  // With the launch's per-camera table, the column term (centre + s_i u) 2^36
  // and the row term (t_j v) 2^36 were rounded on the host exactly as below;
  // one addition and the rounding to the lattice remain per ray.
  long long X[3];
  int D[3], aD[3];
  if (cam.st) {
    const double* col = cam.st + 3 * (size_t)i;
    const double* row = cam.st + 3 * ((size_t)cam.nx + j);
#pragma unroll
    for (int a = 0; a < 3; ++a) X[a] = __double2ll_rn(__dadd_rn(__ldg(col + a), __ldg(row + a)));
  } else {
    const double s = __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn((double)i, 0.5), cam.nxd), 0.5), cam.fov0);
    const double t = __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn((double)j, 0.5), cam.nyd), 0.5), cam.fov1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double x = __dadd_rn(__dadd_rn(cam.centre[a], __dmul_rn(s, cam.u[a])), __dmul_rn(t, cam.v[a]));
      X[a] = __double2ll_rn(__dmul_rn(x, 68719476736.0 /* 2^36 */));
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    D[a] = cam.D[a];
    aD[a] = D[a] < 0 ? -D[a] : D[a];
  }

  // ---- box entry (latest entry time) and exit (earliest exit time) ----------
  // An event is a ray parameter t = num / den, den = |D_axis| > 0.
  bool miss = false;
  long long m = 0, xo = 0;
  int dA = 0, dO = 0, ea = 0;
  bool first = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (D[a] == 0) {
      miss |= (X[a] < 0) | (X[a] >= kBox);
      continue;
    }
    const long long en = D[a] > 0 ? -X[a] : X[a] - kBox;
    const long long ex = D[a] > 0 ? kBox - X[a] : X[a];
    if (first) {
      m = en; dA = aD[a]; ea = a; xo = ex; dO = aD[a];
      first = false;
    } else {
      if (en * dA > m * aD[a]) { m = en; dA = aD[a]; ea = a; }
      if (ex * dO < xo * aD[a]) { xo = ex; dO = aD[a]; }
    }
  }
  if (!miss) miss = !(m * dO < xo * dA);
  if (miss) return res;

  int L = cam.L;
  const uint2* __restrict__ rec = A.rec;
  const void* rho_base = cam.rho;
  const void* v0 = cam.vel[0];
  const void* v1 = cam.vel[1];
  const void* v2 = cam.vel[2];
  int s0 = D[0] > 0 ? 1 : -1, s1 = D[1] > 0 ? 1 : -1, s2 = D[2] > 0 ? 1 : -1;
  // Bit a set: the ray moves down axis a (its cells are entered from the high side).
  const int dirbits = (s0 < 0 ? 1 : 0) | (s1 < 0 ? 2 : 0) | (s2 < 0 ? 4 : 0);

  // ---- descent from the root (Sec. 2.2) ------------------------------------
  uint32_t stack[kMaxLevel + 2];
  uint32_t o = 0;
  uint2 r = __ldg(&rec[0]);
  stack[1] = 0;
  int lvl = 1;
  int k0 = 0, k1 = 0, k2 = 0;
  int c = 0;
  bool bad = false;

  // Walk down from oct o (level q) to the leaf holding the ray just after the
  // entry event (m / dA on axis ea).  Levels q <= lref take the cell from the
  // known coordinates kk (level lref); deeper levels decide each axis by the
  // exact side of the parent cell's mid-plane.
  auto descend = [&](int q, int lref, int kk0, int kk1, int kk2) {
    for (;;) {
      if (q <= lref) {
        const int d = lref - q;
        k0 = kk0 >> d; k1 = kk1 >> d; k2 = kk2 >> d;
      } else {
        const int sh = kFixBits - q;
        const long long M0 = (long long)(2 * k0 + 1) << sh;
        const long long M1 = (long long)(2 * k1 + 1) << sh;
        const long long M2 = (long long)(2 * k2 + 1) << sh;
        const long long g0 = (X[0] - M0) * dA + m * D[0];
        const long long g1 = (X[1] - M1) * dA + m * D[1];
        const long long g2 = (X[2] - M2) * dA + m * D[2];
        k0 = 2 * k0 + ((g0 > 0) | ((g0 == 0) & (D[0] >= 0)));
        k1 = 2 * k1 + ((g1 > 0) | ((g1 == 0) & (D[1] >= 0)));
        k2 = 2 * k2 + ((g2 > 0) | ((g2 == 0) & (D[2] >= 0)));
      }
      c = (k0 & 1) | ((k1 & 1) << 1) | ((k2 & 1) << 2);
      if (!((r.y >> c) & 1u) || q >= L) break;
      const uint32_t ch = r.x + __popc(r.y & ((1u << c) - 1u));
      if (ch >= A.n_oct) { bad = true; break; }  // o still names the oct holding the bad index
      o = ch;
      ++q;
      if (!NB) stack[q] = o;
      r = __ldg(&rec[o]);
    }
    lvl = q;
  };

  // Exact pairwise order of the current cell's exit times t_x = n_x / |D_x|:
  //   e_xy = n_x |D_y| - n_y |D_x|   (the sign of t_x - t_y),
  // with n_x the distance (2^-36 units) from the origin to the cell's exit
  // plane on axis x (n = 1, |D| = 0 for an axis the ray runs parallel to,
  // which makes its time compare as infinite).  Inside a cell of size s both
  // exit times lie within s / |D| of the entry time, so |e_xy| <= s * 2^23:
  // e = E s + r with 0 <= r < s, E a 32-bit integer, and r fixed while the
  // level holds (a step adds |D| s).  The loop keeps F = 2E + (r > 0): its
  // sign is the sign of e (F == 0 exactly when e == 0), a step adds 2|D|, and
  // E = F >> 1.  The increments for each set of stepped axes come from the
  // camera's table (one load instead of per-axis predicated adds).
  int F01, F02, F12;
  long long r01 = 0, r02 = 0, r12 = 0;                  // remainders (FP64 chords)
  // r and s - r of each pair as floats (FP32 chords), at 2 * pair + (ea < b),
  // and 0 at index 6; a small per-thread array read with one indexed load per step.
  // Entries 8..10 hold the remainders r01, r02, r12 of the current level as
  // exact 32-bit integers (bit patterns; exact from level 4 down, where
  // s <= 2^32) for the incremental descent of the FP32 kernels with links.
  __align__(16) float restv[12];
  restv[6] = 0.0f;
  float sf = 0.0f;                                      // s as a float
  auto recompute = [&]() {
    const int sh = kFixBits - lvl;
    const long long n0 = D[0] > 0 ? ((long long)(k0 + 1) << sh) - X[0] : (D[0] < 0 ? X[0] - ((long long)k0 << sh) : 1);
    const long long n1 = D[1] > 0 ? ((long long)(k1 + 1) << sh) - X[1] : (D[1] < 0 ? X[1] - ((long long)k1 << sh) : 1);
    const long long n2 = D[2] > 0 ? ((long long)(k2 + 1) << sh) - X[2] : (D[2] < 0 ? X[2] - ((long long)k2 << sh) : 1);
    const long long e01 = n0 * aD[1] - n1 * aD[0];
    const long long e02 = n0 * aD[2] - n2 * aD[0];
    const long long e12 = n1 * aD[2] - n2 * aD[1];
    const long long E01 = e01 >> sh, E02 = e02 >> sh, E12 = e12 >> sh;  // floor division by s
    const long long mask = (1LL << sh) - 1;  // e - E s: the low bits (floor division)
    r01 = e01 & mask;
    r02 = e02 & mask;
    r12 = e12 & mask;
    F01 = 2 * (int)E01 + (r01 != 0);
    F02 = 2 * (int)E02 + (r02 != 0);
    F12 = 2 * (int)E12 + (r12 != 0);
    if (NB && PREC != AMR_PREC_FP64) {
      restv[8] = __uint_as_float((uint32_t)r01);
      restv[9] = __uint_as_float((uint32_t)r02);
      restv[10] = __uint_as_float((uint32_t)r12);
    }
    const long long s = 1LL << sh;
    restv[0] = __ll2float_rn(r01); restv[1] = __ll2float_rn(s - r01);
    restv[2] = __ll2float_rn(r02); restv[3] = __ll2float_rn(s - r02);
    restv[4] = __ll2float_rn(r12); restv[5] = __ll2float_rn(s - r12);
    sf = __int_as_float((127 + sh) << 23);
  };

  descend(1, 0, 0, 0, 0);
  recompute();
  // Refinement bits that count at the current level: all of them above the
  // camera's cut, none at it (so the step's leaf test is one bit test).
  uint32_t lmask = lvl < L ? 0xFFu : 0u;
  // The ray's origin and direction are needed again only where the level
  // changes or a step crosses an edge or a corner.  A local copy is read back
  // there, so they are not live (in registers) across the common step; the
  // one-level coarsening reads back |D| alone.
  volatile long long keepX[3];
  volatile int keepD[3], keepA[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    keepX[a] = X[a];
    keepD[a] = D[a];
    keepA[a] = aD[a];
  }
  auto reload = [&]() {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      X[a] = keepX[a];
      D[a] = keepD[a];
      aD[a] = D[a] < 0 ? -D[a] : D[a];
    }
    s0 = D[0] > 0 ? 1 : -1;
    s1 = D[1] > 0 ? 1 : -1;
    s2 = D[2] > 0 ? 1 : -1;
    L = cam.L;
  };
  // The one-level coarsening needs only |D|.
  auto reload_aD = [&]() {
#pragma unroll
    for (int a = 0; a < 3; ++a) aD[a] = keepA[a];
  };

  // ---- accumulators ---------------------------------------------------------
  double Sd = 0.0, Nd = 0.0, Md = 0.0;
  float Sf = 0.0f, cSf = 0.0f, Nf = 0.0f, cNf = 0.0f, Mf = 0.0f;
  int count = 0;

  // With links the step keeps only (o, c); the cell's integer coordinates are
  // rebuilt from the oct's packed corner (after its six links) where a level
  // change or a corner needs them.
  auto load_k = [&]() {
    const unsigned long long pk = __ldg(reinterpret_cast<const unsigned long long*>(A.nbr + (size_t)o * 8 + 6));
    k0 = (int)((pk & 0x1FFFFFull) << 1) | (c & 1);
    k1 = (int)(((pk >> 21) & 0x1FFFFFull) << 1) | ((c >> 1) & 1);
    k2 = (int)(((pk >> 42) & 0x1FFFFFull) << 1) | ((c >> 2) & 1);
  };
  // Every step moves on at least one axis (the exit-face test always selects
  // one), so the loop ends; the cap only guards against a corrupted tree.
  while (count < kStepCap) {
    // 32-bit cell and link indices (n_oct * 8 < 2^31 is checked at load): one
    // 32 x 32 -> 64-bit multiply-add per address instead of 64-bit arithmetic.
    const uint32_t cell = o * 8u + (uint32_t)c;
    // A weighted mean over packed fields reads density and velocity in one load.
    constexpr bool kPacked = PACKED && MODE == AMR_MODE_WMEAN;
    Pack4<F> pq{};
    if (kPacked) pq = load_pack<F>(cam.pack, cell);
    const F rho = kPacked ? pq.x : load_field<F>(rho_base, cell);

    // Exit face(s): the axes whose exit time is the minimum.
    const bool lt01 = F01 < 0, gt01 = F01 > 0;
    const bool lt02 = F02 < 0, gt02 = F02 > 0;
    const bool lt12 = F12 < 0, gt12 = F12 > 0;
    const bool st0 = !gt01 && !gt02;
    const bool st1 = !lt01 && !gt12;
    const bool st2 = !lt02 && !lt12;
    const int b = st0 ? 0 : (st1 ? 1 : 2);

    if (MODE == AMR_MODE_MAX) {
      if (PREC == AMR_PREC_FP64) Md = fmax(Md, (double)rho);
      else Mf = fmaxf(Mf, (float)rho);
    } else {
      // Chord.  The cell was entered through its face on axis ea, at n_ea - s:
      //   (t_exit - t_entry) |D_ea| |D_b| = s |D_b| - e'   (b != ea),
      // e' = n_ea |D_b| - n_b |D_ea| = +-e of the pair.  With e = E s + r this is
      //   (K - 1) s + (s - r),  K = |D_b| - E,  when ea < b  (e' = e),
      //    K s + r,             K = |D_b| + E,  when ea > b  (e' = -e),
      // two non-negative parts (K >= 1, resp. K >= 0, since the chord is > 0).
      // The same axis twice (b == ea) gives (t_exit - t_entry) = s / |D_b|,
      // written as K = |D_b| with no remainder part.  The camera's records for
      // (ea, b) hold K's offset, the factor, where the remainder part is, and
      // selectors that pick z E out of (F01, F02, F12) by multiply-adds (FMA
      // pipe) instead of compares and selects (ALU pipe).
      const int4 pc = __ldg(&cam.chord[ea][b]);
      const int4 ps = __ldg(&cam.chordsel[ea][b]);
      const int K = pc.y + ((F01 * ps.x + F02 * ps.y + F12 * ps.z + ps.w) >> 1);
      if (PREC == AMR_PREC_FP64) {
        const int e2 = kFixBits - lvl;  // s = 2^e2
        const long long rp = sel3(pc.w >> 1, r01, r02, r12);  // pair {0,1} -> 0, {0,2} -> 1, {1,2} -> 2
        const long long rest = pc.w == 6 ? 0 : ((pc.w & 1) ? (1LL << e2) - rp : rp);
        const double len = (double)(((long long)K << e2) + rest) * __ldg(&cam.facD[ea][b]);
        const double wgt = (double)rho * len;
        Sd += wgt;
        if (MODE == AMR_MODE_WMEAN) {
          const double vlos = kPacked ? (double)pq.y * cam.w[0] + (double)pq.z * cam.w[1] + (double)pq.w * cam.w[2]
                                      : (double)load_field<F>(v0, cell) * cam.w[0] +
                                            (double)load_field<F>(v1, cell) * cam.w[1] +
                                            (double)load_field<F>(v2, cell) * cam.w[2];
          Nd += wgt * vlos;
        } else if (MODE == AMR_MODE_LEVEL) {
          Nd += wgt * (double)lvl;
        }
      } else {
        // K s is exact in float (|K| < 2^24, s a power of two); one rounding adds the remainder part.
        const float numf = __fmaf_rn(__int2float_rn(K), sf, restv[pc.w]);
        const float len = __fmul_rn(numf, __int_as_float(pc.x));
        const float wgt = __fmul_rn((float)rho, len);
        if (PREC == AMR_PREC_FP32_KAHAN) kahan_add(Sf, cSf, wgt);
        else Sf = __fadd_rn(Sf, wgt);
        if (MODE == AMR_MODE_WMEAN || MODE == AMR_MODE_LEVEL) {
          const float vlos = MODE == AMR_MODE_LEVEL ? (float)lvl
                             : kPacked ? (float)pq.y * cam.wF[0] + (float)pq.z * cam.wF[1] + (float)pq.w * cam.wF[2]
                                       : (float)load_field<F>(v0, cell) * cam.wF[0] +
                                             (float)load_field<F>(v1, cell) * cam.wF[1] +
                                             (float)load_field<F>(v2, cell) * cam.wF[2];
          const float nv = __fmul_rn(wgt, vlos);
          if (PREC == AMR_PREC_FP32_KAHAN) neumaier_add(Nf, cNf, nv);
          else Nf = __fadd_rn(Nf, nv);
        }
      }
    }
    ++count;
    ea = b;

    // Exit planes of the stepped axes move one cell on (valid while the level holds).
    const int stepbits = (st0 ? 1 : 0) | (st1 ? 2 : 0) | (st2 ? 4 : 0);
    const int4 dF = __ldg(&cam.dF[stepbits]);
    F01 += dF.x; F02 += dF.y; F12 += dF.z;
    const int lvl0 = lvl;
    if (NB) {
      // Neighbour at this level.  A step stays inside the oct when every
      // stepped axis moves from the oct's low cell up or from its high cell down.
      const bool inoct = ((c ^ dirbits) & stepbits) == 0;
      c ^= stepbits;
      // Leaving the oct, the step reads one 8-byte word of the oct's link
      // block (the slot comes with the increments): the same-level oct across
      // the face with its refinement mask and level, the coarser leaf covering
      // that side, -1 where the box ends, or (slot 7, for steps on several axes
      // at once) the corner marker.  A same-level step needs no record load;
      // the first-child index is read only when the ray descends.
      int v = (int)o;
      uint32_t ry = r.y;
      if (!inoct) {
        const int2 lk = __ldg(&A.nbr[o * 8u + (uint32_t)dF.w]);
        v = lk.x;
        ry = (uint32_t)lk.y;
      }
      if ((uint32_t)v < A.n_oct && !(((ry & lmask) >> c) & 1u)) {
        // The common step: the same oct, or a same-level oct, and the next
        // cell a leaf at this cut.  Everything else (negative links, the corner
        // marker, out-of-range indices, a refined next cell) takes one branch.
        r.y = ry;
        o = (uint32_t)v;
        continue;
      }
      if ((uint32_t)v < A.n_oct) {
        // A valid link failed the common test: the neighbour is refined
        // above the cut (lmask is 0xFF exactly while lvl < L).
        r.y = ry;
        o = (uint32_t)v;
        if (PREC != AMR_PREC_FP64) {
          // The exact incremental descent needs only |D| and the cut.
          reload_aD();
          if (lvl >= 4 && aD[0] != 0 && aD[1] != 0 && aD[2] != 0) {
            L = cam.L;
            // Exact incremental descent.  The ray entered this cell through
            // its face on axis ea, so on ea the child is the half next to that
            // face.  On another axis a, with the pair term e = H s' + r' in
            // units of the child size s' (H = 2E + the top bit of r, r' its
            // low bits), the entry point lies in the half the ray reaches
            // first iff the entry time precedes the mid-plane crossing:
            // e_(ea,a) < (2|D_a| - |D_ea|) s', i.e. H < T when ea < a and
            // 2(H + T) + [r' > 0] > 0 when ea > a (e_(ea,a) = -e there).  The
            // child's exit planes are the mid-planes on the first-reached
            // axes: E' = H - (u_x |D_y| - u_y |D_x|), r' the low bits.
            uint32_t R0 = __float_as_uint(restv[8]), R1 = __float_as_uint(restv[9]), R2 = __float_as_uint(restv[10]);
            do {
              const uint32_t ch = __ldg(&rec[o].x) + __popc(r.y & ((1u << c) - 1u));
              if (ch >= A.n_oct) { bad = true; break; }
              o = ch;
              r = __ldg(&rec[o]);
              const int shc = kFixBits - lvl - 1;  // <= 31 from level 4 down
              const int t0 = (int)((R0 >> shc) & 1u), t1 = (int)((R1 >> shc) & 1u), t2 = (int)((R2 >> shc) & 1u);
              const uint32_t low = (1u << shc) - 1u;
              R0 &= low;
              R1 &= low;
              R2 &= low;
              const int H0 = (F01 & ~1) | t0, H1 = (F02 & ~1) | t1, H2 = (F12 & ~1) | t2;
              int u0, u1, u2;
              if (ea == 0) {
                u0 = 1;
                u1 = H0 < 2 * aD[1] - aD[0];
                u2 = H1 < 2 * aD[2] - aD[0];
              } else if (ea == 1) {
                u1 = 1;
                u0 = 2 * (H0 + 2 * aD[0] - aD[1]) + (R0 != 0u) > 0;
                u2 = H2 < 2 * aD[2] - aD[1];
              } else {
                u2 = 1;
                u0 = 2 * (H1 + 2 * aD[0] - aD[2]) + (R1 != 0u) > 0;
                u1 = 2 * (H2 + 2 * aD[1] - aD[2]) + (R2 != 0u) > 0;
              }
              F01 = 2 * (H0 - (u0 * aD[1] - u1 * aD[0])) + (R0 != 0u);
              F02 = 2 * (H1 - (u0 * aD[2] - u2 * aD[0])) + (R1 != 0u);
              F12 = 2 * (H2 - (u1 * aD[2] - u2 * aD[1])) + (R2 != 0u);
              // The first-reached half is the low child when the ray moves up
              // that axis, the high one when it moves down.
              c = dirbits ^ (~(u0 | (u1 << 1) | (u2 << 2)) & 7);
              ++lvl;
            } while (((r.y >> c) & 1u) && lvl < L);
            if (bad) break;
            restv[8] = __uint_as_float(R0);
            restv[9] = __uint_as_float(R1);
            restv[10] = __uint_as_float(R2);
            const uint32_t sN = 1u << (kFixBits - lvl);
            restv[0] = __uint2float_rn(R0); restv[1] = __uint2float_rn(sN - R0);
            restv[2] = __uint2float_rn(R1); restv[3] = __uint2float_rn(sN - R1);
            restv[4] = __uint2float_rn(R2); restv[5] = __uint2float_rn(sN - R2);
            sf = __int_as_float((127 + kFixBits - lvl) << 23);
            lmask = lvl < L ? 0xFFu : 0u;
            continue;
          }
        }
        reload();
      } else if (v == kCornerLink) {
        reload();
        // Several axes at once, leaving the oct (an edge or corner): from the root.
        c ^= stepbits;  // back to the cell the ray leaves
        load_k();
        const int j0 = k0 + (st0 ? s0 : 0);
        const int j1 = k1 + (st1 ? s1 : 0);
        const int j2 = k2 + (st2 ? s2 : 0);
        const unsigned lim = 1u << lvl;
        if ((unsigned)j0 >= lim || (unsigned)j1 >= lim || (unsigned)j2 >= lim) break;
        o = 0;
        r = __ldg(&rec[0]);
        const int sh = kFixBits - lvl;
        const int ka = sel3(ea, j0, j1, j2);
        const long long Xa = sel3(ea, X[0], X[1], X[2]);
        m = sel3(ea, s0, s1, s2) > 0 ? ((long long)ka << sh) - Xa : Xa - ((long long)(ka + 1) << sh);
        dA = sel3(ea, aD[0], aD[1], aD[2]);
        descend(1, lvl, j0, j1, j2);
        if (bad) break;
        if (lvl != lvl0) recompute();
        lmask = lvl < L ? 0xFFu : 0u;
        continue;  // the descent stopped at a leaf or the cut: nothing to enter
      } else {
        if (v == -1) break;
        if (v >= 0) { bad = true; break; }
        // A coarser leaf: an unrefined cell, so nothing to enter after it.
        const int cr = -v - 2;
        if (((uint32_t)cr >> 3) >= A.n_oct) { bad = true; break; }
        const int cv = c;  // the same-level cell the step entered (no oct of that level exists there)
        o = (uint32_t)cr >> 3;
        c = cr & 7;
        r.y = ry;
        lvl = (int)((r.y >> 8) & 31u);
        if (lvl < 1 || lvl >= lvl0) { bad = true; break; }
        if (lvl == lvl0 - 1) {
          reload_aD();
          // One level up, the common case: the coarser leaf is the parent of
          // the cell the step entered, so on each axis its exit plane is that
          // cell's, or one cell of the old size s farther when the cell lies in
          // the half its parent's ray enters first (its index bit differs from
          // the direction bit; never on an axis the ray runs parallel to).
          // With j_a = 1 there, e' = e + s (j_a |D_b| - j_b |D_a|) exactly, so
          // for G = E + j_a |D_b| - j_b |D_a| and the new size 2 s:
          // E' = floor(G / 2), r' = (G & 1) s + r, i.e. F' = G | (F & 1).
          const int nz = (aD[0] != 0 ? 1 : 0) | (aD[1] != 0 ? 2 : 0) | (aD[2] != 0 ? 4 : 0);
          const int J = ~(cv ^ dirbits) & nz;
          const int j0 = J & 1, j1 = (J >> 1) & 1, j2 = J >> 2;
          const int G01 = (F01 >> 1) + j0 * aD[1] - j1 * aD[0];
          const int G02 = (F02 >> 1) + j0 * aD[2] - j2 * aD[0];
          const int G12 = (F12 >> 1) + j1 * aD[2] - j2 * aD[1];
          F01 = G01 | (F01 & 1);
          F02 = G02 | (F02 & 1);
          F12 = G12 | (F12 & 1);
          if (PREC == AMR_PREC_FP64) {
            const int sh = kFixBits - lvl0;
            r01 += (long long)(G01 & 1) << sh;
            r02 += (long long)(G02 & 1) << sh;
            r12 += (long long)(G12 & 1) << sh;
          } else {
            // r grows by s where the dropped bit is 1, s - r otherwise: sums of
            // non-negative values, so no cancellation (one more rounding).
            if (MODE == AMR_MODE_WMEAN || MODE == AMR_MODE_LEVEL) {
              // Computed indices (measured faster for the weighted modes,
              // slower for the others, by how the step's registers fall).
              const int i0 = 1 - (G01 & 1), i1 = 3 - (G02 & 1), i2 = 5 - (G12 & 1);
              restv[i0] = __fadd_rn(restv[i0], sf);
              restv[i1] = __fadd_rn(restv[i1], sf);
              restv[i2] = __fadd_rn(restv[i2], sf);
            } else {
              if (G01 & 1) restv[0] = __fadd_rn(restv[0], sf); else restv[1] = __fadd_rn(restv[1], sf);
              if (G02 & 1) restv[2] = __fadd_rn(restv[2], sf); else restv[3] = __fadd_rn(restv[3], sf);
              if (G12 & 1) restv[4] = __fadd_rn(restv[4], sf); else restv[5] = __fadd_rn(restv[5], sf);
            }
            sf = __fmul_rn(sf, 2.0f);
            // The exact remainders gain s where the dropped bit is 1 (only
            // used from level 4 down, where they fit 32 bits).
            const int sho = kFixBits - lvl0;
            const uint32_t add = sho < 32 ? (1u << sho) : 0u;
            restv[8] = __uint_as_float(__float_as_uint(restv[8]) + ((G01 & 1) ? add : 0u));
            restv[9] = __uint_as_float(__float_as_uint(restv[9]) + ((G02 & 1) ? add : 0u));
            restv[10] = __uint_as_float(__float_as_uint(restv[10]) + ((G12 & 1) ? add : 0u));
          }
        } else {
          reload();
          load_k();
          recompute();
        }
        lmask = 0xFFu;  // coarser than before, so above the cut
        continue;       // the coarser leaf is unrefined: nothing to enter
      }
      if (((r.y >> c) & 1u) && lvl < L) {
        // The neighbour is refined: enter its child oct, go on down.
        // By mid-planes from the cell's coordinates, then the 64-bit terms.
        load_k();
        const int sh = kFixBits - lvl;
        const int ka = sel3(ea, k0, k1, k2);
        const long long Xa = sel3(ea, X[0], X[1], X[2]);
        m = sel3(ea, s0, s1, s2) > 0 ? ((long long)ka << sh) - Xa : Xa - ((long long)(ka + 1) << sh);
        dA = sel3(ea, aD[0], aD[1], aD[2]);
        const uint32_t ch = __ldg(&rec[o].x) + __popc(r.y & ((1u << c) - 1u));
        if (ch >= A.n_oct) { bad = true; break; }
        o = ch;
        r = __ldg(&rec[o]);
        descend(lvl + 1, lvl, k0, k1, k2);
        if (bad) break;
        recompute();
        lmask = lvl < L ? 0xFFu : 0u;
      }
    } else {
      // No links: neighbour by coordinates; leaving [0, 2^lvl) ends the ray.
      const int j0 = k0 + (st0 ? s0 : 0);
      const int j1 = k1 + (st1 ? s1 : 0);
      const int j2 = k2 + (st2 ? s2 : 0);
      const unsigned lim = 1u << lvl;
      if ((unsigned)j0 >= lim || (unsigned)j1 >= lim || (unsigned)j2 >= lim) break;
      const int diff = (k0 ^ j0) | (k1 ^ j1) | (k2 ^ j2);
      k0 = j0; k1 = j1; k2 = j2;
      if (diff == 1) {
        c ^= stepbits;
        if (((r.y >> c) & 1u) && lvl < L) {
          const int sh = kFixBits - lvl;
          const int ka = sel3(ea, k0, k1, k2);
          const long long Xa = sel3(ea, X[0], X[1], X[2]);
          m = sel3(ea, s0, s1, s2) > 0 ? ((long long)ka << sh) - Xa : Xa - ((long long)(ka + 1) << sh);
          dA = sel3(ea, aD[0], aD[1], aD[2]);
          const uint32_t ch = r.x + __popc(r.y & ((1u << c) - 1u));
          if (ch >= A.n_oct) { bad = true; break; }
          o = ch;
          stack[lvl + 1] = o;
          r = __ldg(&rec[o]);
          descend(lvl + 1, lvl, j0, j1, j2);
          if (bad) break;
          recompute();
        }
      } else {
        // From the deepest ancestor both cells share (highest differing bit).
        const int q = lvl - (31 - __clz(diff));
        o = stack[q];
        r = __ldg(&rec[o]);
        const int sh = kFixBits - lvl;
        const int ka = sel3(ea, j0, j1, j2);
        const long long Xa = sel3(ea, X[0], X[1], X[2]);
        m = sel3(ea, s0, s1, s2) > 0 ? ((long long)ka << sh) - Xa : Xa - ((long long)(ka + 1) << sh);
        dA = sel3(ea, aD[0], aD[1], aD[2]);
        descend(q, lvl, j0, j1, j2);
        if (bad) break;
        if (lvl != lvl0) recompute();
      }
    }
  }
  if (count >= kStepCap) atomicExch(&A.q->error, (int)kDevStepCap);
  if (bad) {  // o: the oct whose record or link held the bad index
    atomicExch(&A.q->error, (int)kDevBadOct);
    atomicExch(&A.q->err_oct, (int)o);
  }

  res.count = count;
  res.s = Sd; res.n = Nd; res.m = Md;
  // Compensated FP32 sums as (high, low) pairs whose sum is the value: Kahan's
  // term is subtracted (s - c), Neumaier's added (n + c).
  res.sf = Sf; res.cs = PREC == AMR_PREC_FP32_KAHAN ? -cSf : 0.0f;
  res.nf = Nf; res.cn = PREC == AMR_PREC_FP32_KAHAN ? cNf : 0.0f;
  res.mf = Mf;
  return res;
}

// Finalise a ray (wmean = N / S, 0 on an empty ray) and store it, or, for a
// partial render (a sort-last domain's share, Sec. 3.1), store the
// accumulators themselves so that domains can be merged later.
template <int PREC, int MODE, bool PARTIAL>
__device__ __forceinline__ void store_pixel(const CamDev& cam, size_t px, const RayOut& o) {
  constexpr bool weighted = MODE == AMR_MODE_WMEAN || MODE == AMR_MODE_LEVEL;
  if (PARTIAL) {
    if (PREC == AMR_PREC_FP64) {
      if (weighted) static_cast<double2*>(cam.map)[px] = make_double2(o.s, o.n);
      else static_cast<double*>(cam.map)[px] = MODE == AMR_MODE_MAX ? o.m : o.s;
    } else {
      if (weighted) static_cast<float4*>(cam.map)[px] = make_float4(o.sf, o.cs, o.nf, o.cn);
      else if (MODE == AMR_MODE_MAX) static_cast<float*>(cam.map)[px] = o.mf;
      else static_cast<float2*>(cam.map)[px] = make_float2(o.sf, o.cs);
    }
  } else if (PREC == AMR_PREC_FP64) {
    double v = MODE == AMR_MODE_MAX ? o.m : o.s;
    if (weighted) v = o.s != 0.0 ? o.n / o.s : 0.0;
    static_cast<double*>(cam.map)[px] = v;
  } else {
    float v = o.mf;
    if (MODE != AMR_MODE_MAX) {
      const float S = __fadd_rn(o.sf, o.cs);
      v = S;
      if (weighted) v = S != 0.0f ? __fdiv_rn(__fadd_rn(o.nf, o.cn), S) : 0.0f;
    }
    static_cast<float*>(cam.map)[px] = v;
  }
}

template <int PREC, int MODE, bool NB, typename F, bool PARTIAL, bool PACKED = false>
__device__ __forceinline__ int render_mode(const BatchArgs& A, const CamDev& cam, int i, int j) {
  const RayOut o = trace_ray<PREC, MODE, NB, F, PACKED>(A, cam, i, j);
  const size_t px = (size_t)j * cam.nx + i;
  store_pixel<PREC, MODE, PARTIAL>(cam, px, o);
  if (cam.counts) cam.counts[px] = o.count;
  return o.count;
}

template <int PREC, bool NB, typename F, bool PARTIAL>
__device__ __forceinline__ int render_pixel(const BatchArgs& A, const CamDev& cam, int i, int j) {
  switch (cam.mode) {
    case AMR_MODE_COLUMN: return render_mode<PREC, AMR_MODE_COLUMN, NB, F, PARTIAL>(A, cam, i, j);
    case AMR_MODE_WMEAN:
      if (cam.pack) return render_mode<PREC, AMR_MODE_WMEAN, NB, F, PARTIAL, true>(A, cam, i, j);
      return render_mode<PREC, AMR_MODE_WMEAN, NB, F, PARTIAL>(A, cam, i, j);
    case AMR_MODE_LEVEL: return render_mode<PREC, AMR_MODE_LEVEL, NB, F, PARTIAL>(A, cam, i, j);
    default: return render_mode<PREC, AMR_MODE_MAX, NB, F, PARTIAL>(A, cam, i, j);
  }
}

// Persistent batch kernel: each warp repeatedly takes `tiles_per_grab` ray tiles
// from the queue head; a tile index is mapped to its camera by binary search
// over the per-camera tile prefix sums.
// REGS caps the registers per thread.  The default, 64, keeps 32 warps
// resident per SM with 128-thread blocks; the values only the level changes
// and edge crossings use (the ray's origin and direction, the cut) are read
// back from a local copy there, so the common step runs without spills at this
// cap.  56 (36 warps) and 72 (28 warps) are launch options for the map-output
// kernels with links, which the autotuner times per workload.
template <int PREC, bool NB, typename F, bool PARTIAL, int REGS = kDefaultRegs>
__global__ void __maxnreg__(REGS) batch_kernel(const BatchArgs A) {
  const int lane = threadIdx.x & 31;
  unsigned long long segs = 0;
  for (;;) {
    int t0 = 0;
    if (lane == 0) t0 = atomicAdd(&A.q->head, A.tiles_per_grab);
    t0 = __shfl_sync(0xffffffffu, t0, 0);
    if (t0 >= A.total_tiles) break;
    const int t1 = min(t0 + A.tiles_per_grab, A.total_tiles);
    for (int t = t0; t < t1; ++t) {
      int lo = 0, hi = A.n_cams;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&A.tile_start[mid]) <= t) lo = mid;
        else hi = mid;
      }
      const CamDev& cam = A.cams[lo];
      const int lt = t - __ldg(&A.tile_start[lo]) + cam.tile0;
      const int tiles_x = cam.tiles_x;
      const int tx = lt % tiles_x, ty = lt / tiles_x;
      const int i = tx * A.tile_w + lane % A.tile_w;
      const int j = ty * A.tile_h + lane / A.tile_w;
      if (i < cam.nx && j < cam.ny) segs += (unsigned)render_pixel<PREC, NB, F, PARTIAL>(A, cam, i, j);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) segs += __shfl_down_sync(0xffffffffu, segs, off);
  if (lane == 0 && segs) atomicAdd(&A.q->segments, segs);
}

}  // namespace
}  // namespace amr
