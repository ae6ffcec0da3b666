// Octree-AMR ray casting kernels for sm_103a.
//
// One thread traces one pixel ray (Sec. 2.2: "for each pixel of the image, one
// ray is shot").  Warps take 2-D pixel tiles from a device work queue shared by
// every camera of a batch (Sec. 3.2: a master hands work to whichever worker is
// free), so uneven cameras keep every SM busy until the last tile.
//
// Per ray:
//   set-up  : pixel centre in IEEE double (the only FP64 step of the FP32
//             kernels), rounded to the 2^-36 lattice; box entry by exact
//             comparisons of rational crossing times.
//   descent : top-down from the root to the leaf holding the ray (Sec. 2.2),
//             choosing children by the exact side of the mid-planes at the
//             entry time; stops at a leaf or at the camera's level (Sec. 2).
//   step    : the exit face(s) of the current leaf are the earliest crossing
//             times, compared by exact 64-bit cross-multiplication; the chord is
//             the exact integer time difference times a per-camera factor;
//             value x chord is accumulated; the next cell is reached by going
//             up to the deepest oct shared with the neighbour (highest set bit
//             of old xor new integer coordinates) and descending again.
//
// Oct records are 8 bytes {index of the first child oct, 8-bit refinement
// mask}; siblings are contiguous, so the child of cell c is
// first + popc(mask & ((1 << c) - 1)).  Field values are one array per field,
// indexed oct * 8 + cell.
#include "amr_internal.h"
#include "amr.h"

namespace amr {
namespace {

constexpr long long kBox = 1LL << kFixBits;
constexpr int kStepCap = 1 << 25;  // no ray at level <= 22 visits this many leaves

__device__ __forceinline__ int cmp64(long long a, long long b) { return (a > b) - (a < b); }

template <typename T>
__device__ __forceinline__ T sel3(int i, T a, T b, T c) { return i == 0 ? a : (i == 1 ? b : c); }

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

struct RayOut {
  double d;
  float f;
  int count;
};

template <int PREC, int MODE, typename F>
__device__ __forceinline__ RayOut trace_ray(const BatchArgs& A, const CamDev& cam, int i, int j) {
  RayOut res{0.0, 0.0f, 0};

  // ---- ray set-up: FP64 pixel centre, quantised origin ----------------------
  const double s = __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn((double)i, 0.5), cam.nxd), 0.5), cam.fov0);
  const double t = __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn((double)j, 0.5), cam.nyd), 0.5), cam.fov1);
  long long X[3];
  int D[3], aD[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = __dadd_rn(__dadd_rn(cam.centre[a], __dmul_rn(s, cam.u[a])), __dmul_rn(t, cam.v[a]));
    X[a] = __double2ll_rn(__dmul_rn(x, 68719476736.0 /* 2^36 */));
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

  const int L = cam.L;
  const uint2* __restrict__ rec = A.rec;
  const void* rho_base = cam.rho;
  const void* v0 = cam.vel[0];
  const void* v1 = cam.vel[1];
  const void* v2 = cam.vel[2];
  const double lamInv0 = cam.lamInv[0], lamInv1 = cam.lamInv[1], lamInv2 = cam.lamInv[2];
  const double invD0 = cam.invD[0], invD1 = cam.invD[1], invD2 = cam.invD[2];
  const float lamInvF0 = cam.lamInvF[0], lamInvF1 = cam.lamInvF[1], lamInvF2 = cam.lamInvF[2];
  const float invDF0 = cam.invDF[0], invDF1 = cam.invDF[1], invDF2 = cam.invDF[2];
  const int s0 = D[0] > 0 ? 1 : -1, s1 = D[1] > 0 ? 1 : -1, s2 = D[2] > 0 ? 1 : -1;

  double eA = sel3(ea, lamInv0, lamInv1, lamInv2);     // lam / |D| of the entry axis
  float eAF = sel3(ea, lamInvF0, lamInvF1, lamInvF2);

  // ---- top-down descent (Sec. 2.2) -----------------------------------------
  uint32_t stack[kMaxLevel + 2];
  uint32_t o = 0;
  uint2 r = __ldg(&rec[0]);
  stack[1] = 0;
  int lvl = 1;
  int k0 = 0, k1 = 0, k2 = 0;
  int c = 0;
  bool bad = false;

  // Walk down from oct o (level q) to the leaf holding the ray just after the
  // current entry event.  Levels q <= lref take the cell from the known
  // coordinates kk (level lref); deeper levels decide each axis by the exact
  // side of the parent cell's mid-plane.
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
      o = r.x + __popc(r.y & ((1u << c) - 1u));
      if (o >= A.n_oct) { bad = true; break; }
      ++q;
      stack[q] = o;
      r = __ldg(&rec[o]);
    }
    lvl = q;
  };

  descend(1, 0, 0, 0, 0);

  // ---- accumulators ---------------------------------------------------------
  double Sd = 0.0, Nd = 0.0, Md = 0.0;
  float Sf = 0.0f, cSf = 0.0f, Nf = 0.0f, cNf = 0.0f, Mf = 0.0f;
  int count = 0;
  const float wf0 = cam.wF[0], wf1 = cam.wF[1], wf2 = cam.wF[2];
  const double wd0 = cam.w[0], wd1 = cam.w[1], wd2 = cam.w[2];

  while (!bad) {
    const size_t cell = (size_t)o * 8 + c;
    const F rho = load_field<F>(rho_base, cell);

    // Exit event of cell k (level lvl): earliest face crossing ahead of the ray.
    const int sh = kFixBits - lvl;
    const long long n0 = D[0] > 0 ? ((long long)(k0 + 1) << sh) - X[0] : (D[0] < 0 ? X[0] - ((long long)k0 << sh) : 1);
    const long long n1 = D[1] > 0 ? ((long long)(k1 + 1) << sh) - X[1] : (D[1] < 0 ? X[1] - ((long long)k1 << sh) : 1);
    const long long n2 = D[2] > 0 ? ((long long)(k2 + 1) << sh) - X[2] : (D[2] < 0 ? X[2] - ((long long)k2 << sh) : 1);
    // An axis with D = 0 has n = 1 and |D| = 0: its time compares as +infinity.
    const int c01 = cmp64(n0 * aD[1], n1 * aD[0]);
    const long long nw = c01 <= 0 ? n0 : n1;
    const int aw = c01 <= 0 ? aD[0] : aD[1];
    const int mw = c01 < 0 ? 1 : (c01 > 0 ? 2 : 3);
    const int c2 = cmp64(nw * aD[2], n2 * aw);
    const int step = c2 < 0 ? mw : (c2 == 0 ? (mw | 4) : 4);   // axes crossed together
    const int b = c2 > 0 ? 2 : (c01 <= 0 ? 0 : 1);              // exit axis
    const long long nb = c2 > 0 ? n2 : nw;
    const int db = c2 > 0 ? aD[2] : aw;

    // Chord: exact (t_exit - t_entry) |D_b| |D_a|, times lam / (|D_a| |D_b|).
    const long long num = nb * dA - m * db;

    if (MODE == AMR_MODE_MAX) {
      if (PREC == AMR_PREC_FP64) Md = fmax(Md, (double)rho);
      else Mf = fmaxf(Mf, (float)rho);
    } else if (PREC == AMR_PREC_FP64) {
      const double len = (double)num * (eA * sel3(b, invD0, invD1, invD2));
      const double wgt = (double)rho * len;
      Sd += wgt;
      if (MODE == AMR_MODE_WMEAN) {
        const double vlos = (double)load_field<F>(v0, cell) * wd0 + (double)load_field<F>(v1, cell) * wd1 +
                            (double)load_field<F>(v2, cell) * wd2;
        Nd += wgt * vlos;
      }
    } else {
      const float len = __fmul_rn(__ll2float_rn(num), __fmul_rn(eAF, sel3(b, invDF0, invDF1, invDF2)));
      const float wgt = __fmul_rn((float)rho, len);
      if (PREC == AMR_PREC_FP32_KAHAN) kahan_add(Sf, cSf, wgt);
      else Sf = __fadd_rn(Sf, wgt);
      if (MODE == AMR_MODE_WMEAN) {
        const float vlos = (float)load_field<F>(v0, cell) * wf0 + (float)load_field<F>(v1, cell) * wf1 +
                           (float)load_field<F>(v2, cell) * wf2;
        const float nv = __fmul_rn(wgt, vlos);
        if (PREC == AMR_PREC_FP32_KAHAN) neumaier_add(Nf, cNf, nv);
        else Nf = __fadd_rn(Nf, nv);
      }
    }
    ++count;

    // The exit becomes the next entry event.
    m = nb;
    dA = db;
    eA = sel3(b, lamInv0, lamInv1, lamInv2);
    eAF = sel3(b, lamInvF0, lamInvF1, lamInvF2);

    // Neighbour at this level; leaving [0, 2^lvl) on any axis ends the ray.
    const int j0 = k0 + ((step & 1) ? s0 : 0);
    const int j1 = k1 + ((step & 2) ? s1 : 0);
    const int j2 = k2 + ((step & 4) ? s2 : 0);
    const unsigned lim = 1u << lvl;
    if ((unsigned)j0 >= lim || (unsigned)j1 >= lim || (unsigned)j2 >= lim) break;
    // Deepest oct holding both cells: highest differing coordinate bit.
    const int h = 31 - __clz((k0 ^ j0) | (k1 ^ j1) | (k2 ^ j2));
    const int q = lvl - h;
    if (h > 0) {
      o = stack[q];
      r = __ldg(&rec[o]);
    }
    descend(q, lvl, j0, j1, j2);
    if (count >= kStepCap) {
      atomicExch(&A.q->error, (int)kDevStepCap);
      break;
    }
  }
  if (bad) {
    atomicExch(&A.q->error, (int)kDevBadOct);
    atomicExch(&A.q->err_oct, (int)o);
  }

  res.count = count;
  if (PREC == AMR_PREC_FP64) {
    if (MODE == AMR_MODE_COLUMN) res.d = Sd;
    else if (MODE == AMR_MODE_WMEAN) res.d = Sd != 0.0 ? Nd / Sd : 0.0;
    else res.d = Md;
  } else {
    if (MODE == AMR_MODE_COLUMN) {
      res.f = PREC == AMR_PREC_FP32_KAHAN ? __fsub_rn(Sf, cSf) : Sf;
    } else if (MODE == AMR_MODE_WMEAN) {
      const float S = PREC == AMR_PREC_FP32_KAHAN ? __fsub_rn(Sf, cSf) : Sf;
      const float N = PREC == AMR_PREC_FP32_KAHAN ? __fadd_rn(Nf, cNf) : Nf;
      res.f = S != 0.0f ? __fdiv_rn(N, S) : 0.0f;
    } else {
      res.f = Mf;
    }
  }
  return res;
}

template <int PREC, typename F>
__device__ __forceinline__ int render_pixel(const BatchArgs& A, const CamDev& cam, int i, int j) {
  RayOut o;
  switch (cam.mode) {
    case AMR_MODE_COLUMN: o = trace_ray<PREC, AMR_MODE_COLUMN, F>(A, cam, i, j); break;
    case AMR_MODE_WMEAN: o = trace_ray<PREC, AMR_MODE_WMEAN, F>(A, cam, i, j); break;
    default: o = trace_ray<PREC, AMR_MODE_MAX, F>(A, cam, i, j); break;
  }
  const size_t px = (size_t)j * cam.nx + i;
  if (PREC == AMR_PREC_FP64) static_cast<double*>(cam.map)[px] = o.d;
  else static_cast<float*>(cam.map)[px] = o.f;
  if (cam.counts) cam.counts[px] = o.count;
  return o.count;
}

// Persistent batch kernel: each warp repeatedly takes `tiles_per_grab` ray tiles
// from the queue head; a tile index is mapped to its camera by binary search
// over the per-camera tile prefix sums.
template <int PREC, typename F>
__global__ void __launch_bounds__(256) batch_kernel(const BatchArgs A) {
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
      const int lt = t - __ldg(&A.tile_start[lo]);
      const int tiles_x = cam.tiles_x;
      const int tx = lt % tiles_x, ty = lt / tiles_x;
      const int i = tx * A.tile_w + lane % A.tile_w;
      const int j = ty * A.tile_h + lane / A.tile_w;
      if (i < cam.nx && j < cam.ny) segs += (unsigned)render_pixel<PREC, F>(A, cam, i, j);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) segs += __shfl_down_sync(0xffffffffu, segs, off);
  if (lane == 0 && segs) atomicAdd(&A.q->segments, segs);
}

template <int PREC, typename F>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&batch_kernel<PREC, F>);
}

const void* pick(int prec, bool f64) {
  if (f64) {
    switch (prec) {
      case AMR_PREC_FP64: return kernel_ptr<AMR_PREC_FP64, double>();
      case AMR_PREC_FP32_KAHAN: return kernel_ptr<AMR_PREC_FP32_KAHAN, double>();
      default: return kernel_ptr<AMR_PREC_FP32_PLAIN, double>();
    }
  }
  switch (prec) {
    case AMR_PREC_FP64: return kernel_ptr<AMR_PREC_FP64, float>();
    case AMR_PREC_FP32_KAHAN: return kernel_ptr<AMR_PREC_FP32_KAHAN, float>();
    default: return kernel_ptr<AMR_PREC_FP32_PLAIN, float>();
  }
}

}  // namespace

cudaError_t launch_batch(int prec, bool f64, const BatchArgs& a, int grid, int block, cudaStream_t s) {
  void* args[] = {const_cast<BatchArgs*>(&a)};
  return cudaLaunchKernel(pick(prec, f64), dim3(grid), dim3(block), args, 0, s);
}

cudaError_t batch_occupancy(int prec, bool f64, int block, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pick(prec, f64), block, 0);
}

int batch_regs(int prec, bool f64) {
  cudaFuncAttributes at{};
  if (cudaFuncGetAttributes(&at, pick(prec, f64)) != cudaSuccess) return -1;
  return at.numRegs;
}

}  // namespace amr
