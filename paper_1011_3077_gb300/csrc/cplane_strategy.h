// Host-side strategy of the complex-plane recursion (Sec. 3.3): the region
// of a node (a disk cut by half-planes found empty), its enclosing circle, the
// line of each attempt and the per-node decisions (chop, the 2-step rule,
// recentering, giving up).  Plain C++17 with no CUDA dependency, so the same
// code runs in the library's driver and in a CPU test harness.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace eigdc {

struct HalfPlane {
  double wr, wi, t;   // {z : Re(conj(w) z) >= t}
};

struct Region {
  double cr = 0.0, ci = 0.0, R = 0.0;
  std::vector<HalfPlane> hp;
  bool contains(double zr, double zi, double slack = 1e-12) const {
    const double tol = slack * std::max({R, std::hypot(cr, ci), 1e-300});
    if (std::hypot(zr - cr, zi - ci) > R + tol) return false;
    for (const HalfPlane& h : hp)
      if (h.wr * zr + h.wi * zi < h.t - tol) return false;
    return true;
  }
};

struct Pt {
  double x, y;
};

inline void line_circle(const Region& g, const HalfPlane& h, std::vector<Pt>& out) {
  const double d = h.t - (h.wr * g.cr + h.wi * g.ci);
  if (std::fabs(d) > g.R) return;
  const double hh = std::sqrt(std::max(g.R * g.R - d * d, 0.0));
  const double fx = g.cr + h.wr * d, fy = g.ci + h.wi * d;
  // i w = (-wi, wr)
  out.push_back({fx - h.wi * hh, fy + h.wr * hh});
  out.push_back({fx + h.wi * hh, fy - h.wr * hh});
}

inline bool line_line(const HalfPlane& a, const HalfPlane& b, Pt* p) {
  const double det = a.wr * b.wi - a.wi * b.wr;
  if (std::fabs(det) < 1e-14) return false;
  p->x = (a.t * b.wi - a.wi * b.t) / det;
  p->y = (a.wr * b.t - a.t * b.wr) / det;
  return true;
}

inline bool circle3(Pt p, Pt q, Pt r, Pt* m, double* rad) {
  const double d = 2.0 * (p.x * (q.y - r.y) + q.x * (r.y - p.y) + r.x * (p.y - q.y));
  if (std::fabs(d) < 1e-300) return false;
  const double pp = p.x * p.x + p.y * p.y, qq = q.x * q.x + q.y * q.y, rr = r.x * r.x + r.y * r.y;
  m->x = (pp * (q.y - r.y) + qq * (r.y - p.y) + rr * (p.y - q.y)) / d;
  m->y = (pp * (r.x - q.x) + qq * (p.x - r.x) + rr * (q.x - p.x)) / d;
  *rad = std::hypot(p.x - m->x, p.y - m->y);
  return true;
}

// Smallest circle through a few points: every pair as a diameter and every
// triple's circumcircle, the smallest that holds all points.
inline bool min_circle(const std::vector<Pt>& pts, Pt* m, double* rad) {
  if (pts.empty()) return false;
  if (pts.size() == 1) {
    *m = pts[0];
    *rad = 0.0;
    return true;
  }
  bool have = false;
  auto consider = [&](Pt c, double r) {
    const double tol = 1e-12 * std::max(r, 1e-300);
    for (const Pt& p : pts)
      if (std::hypot(p.x - c.x, p.y - c.y) > r + tol) return;
    if (!have || r < *rad) {
      have = true;
      *m = c;
      *rad = r;
    }
  };
  const size_t np = pts.size();
  for (size_t i = 0; i < np; ++i)
    for (size_t j = i + 1; j < np; ++j) {
      consider({0.5 * (pts[i].x + pts[j].x), 0.5 * (pts[i].y + pts[j].y)},
               0.5 * std::hypot(pts[i].x - pts[j].x, pts[i].y - pts[j].y));
      for (size_t k = j + 1; k < np; ++k) {
        Pt c;
        double r;
        if (circle3(pts[i], pts[j], pts[k], &c, &r)) consider(c, r);
      }
    }
  return have;
}

// Circle holding the region: the smallest circle through its corners when it
// also holds the boundary arc (the point of the circle opposite its centre,
// if that point is in the region); otherwise the disk itself.
inline void enclosing_circle(const Region& g, double* mr, double* mi, double* rad) {
  *mr = g.cr;
  *mi = g.ci;
  *rad = g.R;
  if (g.hp.empty()) return;
  std::vector<Pt> corners, tmp;
  for (size_t i = 0; i < g.hp.size(); ++i) {
    tmp.clear();
    line_circle(g, g.hp[i], tmp);
    for (const Pt& p : tmp)
      if (g.contains(p.x, p.y)) corners.push_back(p);
    for (size_t j = i + 1; j < g.hp.size(); ++j) {
      Pt p;
      if (line_line(g.hp[i], g.hp[j], &p) && g.contains(p.x, p.y)) corners.push_back(p);
    }
  }
  Pt m{0.0, 0.0};
  double r = 0.0;
  if (!min_circle(corners, &m, &r)) return;
  if (r >= g.R || (m.x == g.cr && m.y == g.ci)) return;
  const double dx = m.x - g.cr, dy = m.y - g.ci, dn = std::hypot(dx, dy);
  const double fx = g.cr - g.R * dx / dn, fy = g.ci - g.R * dy / dn;
  if (g.contains(fx, fy) && std::hypot(fx - m.x, fy - m.y) > r * (1.0 + 1e-12)) return;
  *mr = m.x;
  *mi = m.y;
  *rad = r;
}

// The line of an attempt from its two uniforms: angle 2 pi u2, or the
// perpendicular i w' of the previous chord's normal w' = (pr, pi); offset
// R (u1 - 1/2) from the centre along the normal.
inline HalfPlane make_line(const Region& g, double u1, double u2, bool has_perp, double pr,
                           double pi_) {
  HalfPlane h;
  if (has_perp) {
    h.wr = -pi_;   // i w
    h.wi = pr;
  } else {
    const double th = 2.0 * 3.14159265358979323846 * u2;
    h.wr = std::cos(th);
    h.wi = std::sin(th);
  }
  const double a = g.R * (u1 - 0.5);
  h.t = a + (h.wr * g.cr + h.wi * g.ci);
  return h;
}

constexpr double CPLANE_SHRINK = 0.96592582628906829;   // sin(5 pi / 12)

// Per-node decisions of the Sec. 3.3 strategy after a step that did not split.
struct NodePlan {
  Region reg;
  int attempt = 0, fails = 0;
  bool has_perp = false;
  double pr = 0.0, pi_ = 0.0;
  int max_fail = 8, max_attempts = 250;
  // recentering log of the last call: 0 none, 1 after one chop, 2 after two
  int recentered = 0;
  double old_R = 0.0;

  HalfPlane line(double u1, double u2) const { return make_line(reg, u1, u2, has_perp, pr, pi_); }

  // The step on line L converged with RURV rank `rank` of m (a chop when it is
  // 0 or m) or failed.  Returns true when the node gives up (a cluster).
  bool after_nonsplit(const HalfPlane& L, bool converged, int rank, int m) {
    recentered = 0;
    if (converged && (rank == 0 || rank == m)) {
      reg.hp.push_back(rank == m ? L : HalfPlane{-L.wr, -L.wi, -L.t});
      double er, ei, eR;
      enclosing_circle(reg, &er, &ei, &eR);
      if (eR <= CPLANE_SHRINK * reg.R) {
        old_R = reg.R;
        reg = Region();
        reg.cr = er;
        reg.ci = ei;
        reg.R = eR;
        recentered = 1;
        has_perp = false;
      } else if (!has_perp) {
        has_perp = true;
        pr = L.wr;
        pi_ = L.wi;
      } else {
        if (eR < reg.R) {
          old_R = reg.R;
          reg = Region();
          reg.cr = er;
          reg.ci = ei;
          reg.R = eR;
          recentered = 2;
        }
        has_perp = false;
      }
    } else {
      fails += 1;
      has_perp = false;
    }
    attempt += 1;
    return fails > max_fail || attempt > max_attempts;
  }
};

// Regions of the two blocks after a split on L: each side's enclosing circle,
// or the block's own disk (about its mean eigenvalue, radius ||A_ii - cI||_F)
// when that is not larger.
inline void child_regions(const Region& reg, const HalfPlane& L, const Region* gersh0,
                          const Region* gersh1, Region* kid0, Region* kid1) {
  Region sides[2] = {reg, reg};
  sides[0].hp.push_back(L);
  sides[1].hp.push_back({-L.wr, -L.wi, -L.t});
  const Region* g[2] = {gersh0, gersh1};
  Region* out[2] = {kid0, kid1};
  for (int c = 0; c < 2; ++c) {
    double er, ei, eR;
    enclosing_circle(sides[c], &er, &ei, &eR);
    if (g[c] && g[c]->R <= eR) {
      *out[c] = *g[c];
    } else {
      *out[c] = Region();
      out[c]->cr = er;
      out[c]->ci = ei;
      out[c]->R = eR;
    }
  }
}

}  // namespace eigdc
