// Seeded synthetic octree generator.  Input generation only: it decides the
// tree shape and the cell values, and holds none of the ray-casting arithmetic.
//
// Octree model (Sec. 1, Fig. 1 right): RAMSES octs of 8 cells, root oct of
// level 1, refinement to level 22 (Sec. 1 and Fig. 3 caption quote level 22
// and ~200M cells for the Milky-Way run).  The density models, the random
// fields and the refinement rule are readings written down with the workloads:
//   plain  : rho = 1 + 100 exp(-|x-c|^2 / (2*0.05^2)), refine while
//            rho(centre) 8^-l > threshold.
//   galaxy : rho = 1e-6 + exp(-R/0.05) exp(-|z|/0.005) exp(0.5 g) in a disk frame
//            with a seeded normal, g a unit-variance Gaussian random field with
//            P(k) ~ k^-11/3 made of seeded Fourier modes; refine while
//            rho(centre) 8^-l > threshold * (total mass of the base grid).
//            Velocity = flat rotation curve + 0.1 x three more random fields.
//            Optional Plummer clumps make refinement reach level 22.
#include "../../../include/amr_gen.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <omp.h>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxLevel = 22;
// Uniform background density of the galaxy model (1e-6 of the central disk
// density): keeps every float32 density and column far above the float32
// underflow range; the bare exponential disk falls below 1e-38 at |z| ~ 0.44.
constexpr double kBackground = 1e-6;

// splitmix64: a published counter-based mixer (Steele, Lea, Flood 2014).
struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(seed) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0,1)
  double uniform_pos() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }  // (0,1)
  void unit_vector(double out[3]) {
    double z = 2.0 * uniform() - 1.0;
    double phi = 2.0 * kPi * uniform();
    double r = std::sqrt(std::fmax(0.0, 1.0 - z * z));
    out[0] = r * std::cos(phi);
    out[1] = r * std::sin(phi);
    out[2] = z;
  }
};

// One Gaussian random field: g(x) = sum_m a_m cos(k_m . x + phi_m).
// |k| log-uniform in [2pi, 2pi 2^14]; each mode stands for a d(ln k) slice, so
// a_m^2 ~ k^3 P(k) = k^-2/3; normalised so that sum a_m^2 / 2 = 1 (Var g = 1).
struct Grf {
  int m = 0;
  std::vector<double> k;     // [m][3]
  std::vector<double> amp;   // [m]
  std::vector<double> phase; // [m]
  // Per level l: e^{i h_l k_x}, e^{i h_l k_y}, e^{i h_l k_z} with h_l = 2^-l.
  std::vector<double> stepc, steps;  // [(kMaxLevel+1)][m][3]

  void init(Rng& rng, int n_modes) {
    m = n_modes;
    k.resize(3 * m);
    amp.resize(m);
    phase.resize(m);
    double sum2 = 0.0;
    for (int i = 0; i < m; ++i) {
      double kmag = 2.0 * kPi * std::exp2(14.0 * rng.uniform());
      double dir[3];
      rng.unit_vector(dir);
      for (int a = 0; a < 3; ++a) k[3 * i + a] = kmag * dir[a];
      phase[i] = 2.0 * kPi * rng.uniform();
      amp[i] = std::pow(kmag, -1.0 / 3.0);
      sum2 += amp[i] * amp[i];
    }
    double norm = std::sqrt(2.0 / sum2);
    for (int i = 0; i < m; ++i) amp[i] *= norm;
    stepc.resize((kMaxLevel + 1) * m * 3);
    steps.resize((kMaxLevel + 1) * m * 3);
    for (int l = 0; l <= kMaxLevel; ++l) {
      double h = std::ldexp(1.0, -l);
      for (int i = 0; i < m; ++i)
        for (int a = 0; a < 3; ++a) {
          size_t idx = ((size_t)l * m + i) * 3 + a;
          stepc[idx] = std::cos(h * k[3 * i + a]);
          steps[idx] = std::sin(h * k[3 * i + a]);
        }
    }
  }

  double at(const double x[3]) const {
    double g = 0.0;
    for (int i = 0; i < m; ++i)
      g += amp[i] * std::cos(k[3 * i] * x[0] + k[3 * i + 1] * x[1] + k[3 * i + 2] * x[2] + phase[i]);
    return g;
  }

  // Values at the 8 cell centres of an oct whose cell 0 is centred at x0 and
  // whose cells have level l: rotate e^{i theta(x0)} by the per-axis steps.
  void oct(const double x0[3], int l, double out[8]) const {
    for (int c = 0; c < 8; ++c) out[c] = 0.0;
    const double* sc = &stepc[(size_t)l * m * 3];
    const double* ss = &steps[(size_t)l * m * 3];
    for (int i = 0; i < m; ++i) {
      double th = k[3 * i] * x0[0] + k[3 * i + 1] * x0[1] + k[3 * i + 2] * x0[2] + phase[i];
      double c0 = std::cos(th), s0 = std::sin(th);
      double cx = sc[3 * i], sx = ss[3 * i];
      double cy = sc[3 * i + 1], sy = ss[3 * i + 1];
      double cz = sc[3 * i + 2], sz = ss[3 * i + 2];
      double c1 = c0 * cx - s0 * sx, s1 = s0 * cx + c0 * sx;  // +x
      double c2 = c0 * cy - s0 * sy, s2 = s0 * cy + c0 * sy;  // +y
      double c3 = c1 * cy - s1 * sy, s3 = s1 * cy + c1 * sy;  // +x+y
      double a = amp[i];
      out[0] += a * c0;
      out[1] += a * c1;
      out[2] += a * c2;
      out[3] += a * c3;
      out[4] += a * (c0 * cz - s0 * sz);
      out[5] += a * (c1 * cz - s1 * sz);
      out[6] += a * (c2 * cz - s2 * sz);
      out[7] += a * (c3 * cz - s3 * sz);
    }
  }
};

struct Clump {
  double pos[3];
  double a;      // Plummer scale radius
  double mass;
  double rho0;   // 3 M / (4 pi a^3)
};

struct Model {
  amrgen_params p{};
  double normal[3] = {0, 0, 1};
  double e1[3] = {1, 0, 0}, e2[3] = {0, 1, 0};
  Grf g, gv[3];
  std::vector<Clump> clumps;

  void init(const amrgen_params& prm) {
    p = prm;
    if (p.kind != AMRGEN_GALAXY) return;
    Rng rng(p.seed * 0x2545F4914F6CDD1Dull + 0x1234567ull);
    rng.unit_vector(normal);
    // Orthonormal basis of the disk plane.
    double ref[3] = {1, 0, 0};
    if (std::fabs(normal[0]) > 0.9) { ref[0] = 0; ref[1] = 1; }
    cross(normal, ref, e1);
    normalise(e1);
    cross(normal, e1, e2);
    g.init(rng, p.n_modes);
    if (p.with_velocity)
      for (int a = 0; a < 3; ++a) gv[a].init(rng, p.n_modes);
    if (p.n_clumps > 0) {
      // Exponential-disk mass over all space: 4 pi h_R^2 h_z.
      double mdisk = 4.0 * kPi * 0.05 * 0.05 * 0.005;
      for (int j = 0; j <= p.n_clumps; ++j) {
        Clump c;
        double R = 0.0, z = 0.0, ang = 0.0;
        if (j > 0) {
          R = -0.05 * (std::log(rng.uniform_pos()) + std::log(rng.uniform_pos()));  // Gamma(2, 0.05)
          if (R > 0.4) R = 0.4;
          ang = 2.0 * kPi * rng.uniform();
          double e = -0.005 * std::log(rng.uniform_pos());
          z = (rng.uniform() < 0.5) ? -e : e;                                      // Laplace(0.005)
        }
        for (int a = 0; a < 3; ++a)
          c.pos[a] = 0.5 + R * (std::cos(ang) * e1[a] + std::sin(ang) * e2[a]) + z * normal[a];
        c.a = std::exp2(-21.0 + 11.0 * rng.uniform());
        c.mass = 1e-4 * mdisk;
        c.rho0 = 3.0 * c.mass / (4.0 * kPi * c.a * c.a * c.a);
        clumps.push_back(c);
      }
    }
  }

  static void cross(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
  }
  static void normalise(double v[3]) {
    double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int a = 0; a < 3; ++a) v[a] /= n;
  }

  double smooth_disk(const double x[3], double gval) const {
    double d[3] = {x[0] - 0.5, x[1] - 0.5, x[2] - 0.5};
    double zz = d[0] * normal[0] + d[1] * normal[1] + d[2] * normal[2];
    double pr[3] = {d[0] - zz * normal[0], d[1] - zz * normal[1], d[2] - zz * normal[2]};
    double R = std::sqrt(pr[0] * pr[0] + pr[1] * pr[1] + pr[2] * pr[2]);
    return kBackground + std::exp(-R / 0.05) * std::exp(-std::fabs(zz) / 0.005) * std::exp(0.5 * gval);
  }

  double clump_density(const double x[3]) const {
    double s = 0.0;
    for (const Clump& c : clumps) {
      double r2 = 0.0;
      for (int a = 0; a < 3; ++a) r2 += (x[a] - c.pos[a]) * (x[a] - c.pos[a]);
      double q = 1.0 + r2 / (c.a * c.a);
      s += c.rho0 / (q * q * std::sqrt(q));
    }
    return s;
  }

  void rotation(const double x[3], double v[3]) const {
    double d[3] = {x[0] - 0.5, x[1] - 0.5, x[2] - 0.5};
    double t[3];
    cross(normal, d, t);  // in the disk plane, |t| = R
    double R = std::sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    if (R == 0.0) { v[0] = v[1] = v[2] = 0.0; return; }
    double vphi = R / std::sqrt(R * R + 0.02 * 0.02);
    for (int a = 0; a < 3; ++a) v[a] = vphi * t[a] / R;
  }

  // Density (smooth part separately) and velocity at the 8 cell centres.
  void eval_oct(int level, const int32_t coord[3], double rho[8], double smooth[8],
                double vel[3][8]) const {
    double h = std::ldexp(1.0, -level);
    double x0[3];
    for (int a = 0; a < 3; ++a) x0[a] = ((double)coord[a] + 0.5) * h;
    if (p.kind == AMRGEN_PLAIN) {
      for (int c = 0; c < 8; ++c) {
        double x[3] = {x0[0] + (c & 1) * h, x0[1] + ((c >> 1) & 1) * h, x0[2] + ((c >> 2) & 1) * h};
        double r2 = 0.0;
        for (int a = 0; a < 3; ++a) r2 += (x[a] - 0.5) * (x[a] - 0.5);
        rho[c] = smooth[c] = 1.0 + 100.0 * std::exp(-r2 / (2.0 * 0.05 * 0.05));
      }
      return;
    }
    double gv8[8];
    g.oct(x0, level, gv8);
    double vv[3][8];
    if (p.with_velocity)
      for (int a = 0; a < 3; ++a) gv[a].oct(x0, level, vv[a]);
    for (int c = 0; c < 8; ++c) {
      double x[3] = {x0[0] + (c & 1) * h, x0[1] + ((c >> 1) & 1) * h, x0[2] + ((c >> 2) & 1) * h};
      smooth[c] = smooth_disk(x, gv8[c]);
      rho[c] = smooth[c] + (clumps.empty() ? 0.0 : clump_density(x));
      if (p.with_velocity) {
        double r[3];
        rotation(x, r);
        for (int a = 0; a < 3; ++a) vel[a][c] = r[a] + 0.1 * vv[a][c];
      }
    }
  }

  // Clump rule: a cell holding a clump centre is refined while the Plummer mass
  // inside the radius h/2 around that centre exceeds the threshold; this lets the
  // mass criterion follow clumps smaller than the cell (point sampling alone
  // would miss them).
  bool clump_refine(int level, const int32_t cellk[3], double thr_abs) const {
    if (clumps.empty()) return false;
    double h = std::ldexp(1.0, -level);
    for (const Clump& c : clumps) {
      bool inside = true;
      for (int a = 0; a < 3; ++a) {
        double lo = cellk[a] * h;
        if (!(c.pos[a] >= lo && c.pos[a] < lo + h)) { inside = false; break; }
      }
      if (!inside) continue;
      double r = 0.5 * h;
      double q = r * r + c.a * c.a;
      double menc = c.mass * r * r * r / (q * std::sqrt(q));
      if (menc > thr_abs) return true;
    }
    return false;
  }
};

}  // namespace

struct amrgen_tree {
  int64_t n_oct = 0;
  int32_t n_fields = 1;
  std::vector<uint8_t> level;
  std::vector<int32_t> coord;
  std::vector<int32_t> child;
  std::vector<double> rho;
  std::vector<double> vel[3];
  double total_mass = 0.0;
  double thr_abs = 0.0;
  double normal[3] = {0, 0, 1};
  int64_t hist[kMaxLevel + 1] = {};
  int64_t n_leaves = 0;
};

extern "C" {

int amrgen_build(const amrgen_params* p, amrgen_tree** out) {
  if (!p || !out) return -1;
  *out = nullptr;
  if (p->kind != AMRGEN_PLAIN && p->kind != AMRGEN_GALAXY) return -1;
  if (p->base_level < 1 || p->max_level < p->base_level || p->max_level > kMaxLevel) return -1;
  if (p->kind == AMRGEN_GALAXY && p->n_modes < 1) return -1;
  amrgen_tree* t = new (std::nothrow) amrgen_tree;
  if (!t) return -3;
  try {
    Model model;
    model.init(*p);
    const bool vel = (p->kind == AMRGEN_GALAXY) && p->with_velocity;
    t->n_fields = vel ? 4 : 1;
    for (int a = 0; a < 3; ++a) t->normal[a] = model.normal[a];
    int nthreads = p->n_threads > 0 ? p->n_threads : omp_get_max_threads();
    std::vector<double> smooth;

    // Root oct.
    t->level.push_back(1);
    t->coord.insert(t->coord.end(), {0, 0, 0});
    t->child.insert(t->child.end(), 8, -1);
    int64_t first = 0, last = 1;  // octs of the current level: [first, last)
    double thr_abs = (p->kind == AMRGEN_PLAIN) ? p->threshold : 0.0;
    for (int lvl = 1; first < last; ++lvl) {
      int64_t n = last - first;
      t->rho.resize((size_t)last * 8);
      smooth.resize((size_t)last * 8);
      if (vel)
        for (int a = 0; a < 3; ++a) t->vel[a].resize((size_t)last * 8);
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
      for (int64_t i = 0; i < n; ++i) {
        int64_t o = first + i;
        double vv[3][8];
        model.eval_oct(lvl, &t->coord[3 * o], &t->rho[8 * o], &smooth[8 * o], vv);
        if (vel)
          for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 8; ++c) t->vel[a][8 * o + c] = vv[a][c];
      }
      if (p->kind == AMRGEN_GALAXY && lvl == p->base_level) {
        // Total mass of the base-level grid (smooth disk part), in cell units.
        double tot = 0.0;
        double vol = std::ldexp(1.0, -3 * lvl);
        for (int64_t o = first; o < last; ++o)
          for (int c = 0; c < 8; ++c) tot += smooth[8 * o + c] * vol;
        t->total_mass = tot;
        thr_abs = p->threshold * tot;
      }
      if (lvl >= p->max_level) break;
      // Refinement decisions, then children in oct order / cell order.
      std::vector<uint8_t> refine((size_t)n * 8, 0);
      double vol = std::ldexp(1.0, -3 * lvl);
#pragma omp parallel for schedule(static) num_threads(nthreads)
      for (int64_t i = 0; i < n; ++i) {
        int64_t o = first + i;
        for (int c = 0; c < 8; ++c) {
          bool r;
          if (lvl < p->base_level) {
            r = true;
          } else {
            r = t->rho[8 * o + c] * vol > thr_abs;
            if (!r) {
              int32_t k[3] = {t->coord[3 * o] + (c & 1), t->coord[3 * o + 1] + ((c >> 1) & 1),
                              t->coord[3 * o + 2] + ((c >> 2) & 1)};
              r = model.clump_refine(lvl, k, thr_abs);
            }
          }
          refine[8 * i + c] = r ? 1 : 0;
        }
      }
      int64_t next = last;
      for (int64_t i = 0; i < n; ++i) {
        int64_t o = first + i;
        for (int c = 0; c < 8; ++c) {
          if (!refine[8 * i + c]) continue;
          t->child[8 * o + c] = (int32_t)next;
          t->level.push_back((uint8_t)(lvl + 1));
          for (int a = 0; a < 3; ++a)
            t->coord.push_back(2 * (t->coord[3 * o + a] + ((c >> a) & 1)));
          t->child.insert(t->child.end(), 8, -1);
          ++next;
        }
      }
      if (next > (int64_t)0x7fffffff) throw std::bad_alloc();
      first = last;
      last = next;
    }
    t->n_oct = (int64_t)t->level.size();
    t->thr_abs = thr_abs;
    // Restriction, finest octs first: a refined cell holds the mean density of
    // its 8 children and their density-weighted mean velocity.
    for (int64_t o = t->n_oct - 1; o >= 0; --o) {
      for (int c = 0; c < 8; ++c) {
        int32_t ch = t->child[8 * o + c];
        if (ch < 0) continue;
        double s = 0.0, sv[3] = {0, 0, 0};
        for (int q = 0; q < 8; ++q) {
          double r = t->rho[8 * (size_t)ch + q];
          s += r;
          if (vel)
            for (int a = 0; a < 3; ++a) sv[a] += r * t->vel[a][8 * (size_t)ch + q];
        }
        t->rho[8 * o + c] = s / 8.0;
        if (vel)
          for (int a = 0; a < 3; ++a) {
            if (s > 0.0) {
              t->vel[a][8 * o + c] = sv[a] / s;
            } else {
              double m = 0.0;
              for (int q = 0; q < 8; ++q) m += t->vel[a][8 * (size_t)ch + q];
              t->vel[a][8 * o + c] = m / 8.0;
            }
          }
      }
    }
    for (int64_t o = 0; o < t->n_oct; ++o)
      for (int c = 0; c < 8; ++c)
        if (t->child[8 * o + c] < 0) {
          t->hist[t->level[o]]++;
          t->n_leaves++;
        }
  } catch (const std::bad_alloc&) {
    delete t;
    return -3;
  }
  *out = t;
  return 0;
}

int64_t amrgen_n_oct(const amrgen_tree* t) { return t ? t->n_oct : -1; }
int32_t amrgen_n_fields(const amrgen_tree* t) { return t ? t->n_fields : -1; }

int amrgen_copy(const amrgen_tree* t, uint8_t* level, int32_t* coord, int32_t* child,
                void* const* fields, int32_t field_dtype) {
  if (!t || (field_dtype != 0 && field_dtype != 1)) return -1;
  size_t n = (size_t)t->n_oct;
  if (level) std::memcpy(level, t->level.data(), n);
  if (coord) std::memcpy(coord, t->coord.data(), n * 3 * sizeof(int32_t));
  if (child) std::memcpy(child, t->child.data(), n * 8 * sizeof(int32_t));
  if (fields) {
    for (int f = 0; f < t->n_fields; ++f) {
      if (!fields[f]) continue;
      const double* src = (f == 0) ? t->rho.data() : t->vel[f - 1].data();
      if (field_dtype == 1) {
        std::memcpy(fields[f], src, n * 8 * sizeof(double));
      } else {
        float* dst = (float*)fields[f];
        for (size_t i = 0; i < n * 8; ++i) dst[i] = (float)src[i];
      }
    }
  }
  return 0;
}

int64_t amrgen_info(const amrgen_tree* t, char* buf, int64_t buf_len) {
  if (!t || !buf || buf_len <= 0) return -1;
  std::string s = "{\"n_oct\": " + std::to_string(t->n_oct) +
                  ", \"n_leaves\": " + std::to_string(t->n_leaves) +
                  ", \"n_fields\": " + std::to_string(t->n_fields);
  char tmp[256];
  std::snprintf(tmp, sizeof tmp, ", \"total_mass\": %.17g, \"threshold_abs\": %.17g", t->total_mass,
                t->thr_abs);
  s += tmp;
  std::snprintf(tmp, sizeof tmp, ", \"normal\": [%.17g, %.17g, %.17g]", t->normal[0], t->normal[1],
                t->normal[2]);
  s += tmp;
  s += ", \"leaf_hist\": {";
  bool firstk = true;
  for (int l = 0; l <= kMaxLevel; ++l) {
    if (!t->hist[l]) continue;
    if (!firstk) s += ", ";
    firstk = false;
    s += "\"" + std::to_string(l) + "\": " + std::to_string(t->hist[l]);
  }
  s += "}}";
  int64_t n = (int64_t)s.size();
  if (n > buf_len - 1) n = buf_len - 1;
  std::memcpy(buf, s.data(), (size_t)n);
  buf[n] = '\0';
  return n;
}

void amrgen_free(amrgen_tree* t) { delete t; }

int amrgen_sample(const amrgen_params* p, int32_t which, int64_t n, const double* xyz, double* out) {
  if (!p || !xyz || !out || which < 0 || which > 4 || n < 0) return -1;
  if (p->kind != AMRGEN_GALAXY && which != 0) return -1;
  if (which >= 2 && !p->with_velocity) return -1;
  Model model;
  model.init(*p);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double* x = xyz + 3 * i;
    double val;
    if (p->kind == AMRGEN_PLAIN) {
      double r2 = 0.0;
      for (int a = 0; a < 3; ++a) r2 += (x[a] - 0.5) * (x[a] - 0.5);
      val = 1.0 + 100.0 * std::exp(-r2 / (2.0 * 0.05 * 0.05));
    } else if (which == 0) {
      val = model.smooth_disk(x, model.g.at(x)) + (model.clumps.empty() ? 0.0 : model.clump_density(x));
    } else if (which == 1) {
      val = model.g.at(x);
    } else {
      double r[3];
      model.rotation(x, r);
      val = r[which - 2] + 0.1 * model.gv[which - 2].at(x);
    }
    out[i] = val;
  }
  return 0;
}

}  // extern "C"
