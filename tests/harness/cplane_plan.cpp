// CPU harness for the library's per-node strategy (cplane_strategy.h): reads
// a node's starting disk and, per attempt, the two line uniforms and the step
// outcome; prints the line and the disk of every attempt and the node's end.
//
// stdin:  R cr ci m max_fail
//         count
//         count lines "u1 u2 kind rank" (kind 0 split, 1 converged no split, 2 failed)
// stdout: "line wr wi t cr ci R" per attempt, then "end split|cluster|open"
#include <cstdio>

#include "cplane_strategy.h"

int main() {
  double R, cr, ci;
  int m, max_fail, count;
  if (std::scanf("%lf %lf %lf %d %d %d", &R, &cr, &ci, &m, &max_fail, &count) != 6) return 2;
  eigdc::NodePlan plan;
  plan.reg.cr = cr;
  plan.reg.ci = ci;
  plan.reg.R = R;
  plan.max_fail = max_fail;
  for (int a = 0; a < count; ++a) {
    double u1, u2;
    int kind, rank;
    if (std::scanf("%lf %lf %d %d", &u1, &u2, &kind, &rank) != 4) return 2;
    const eigdc::HalfPlane L = plan.line(u1, u2);
    std::printf("line %.17g %.17g %.17g %.17g %.17g %.17g\n", L.wr, L.wi, L.t, plan.reg.cr,
                plan.reg.ci, plan.reg.R);
    if (kind == 0) {
      std::printf("end split\n");
      return 0;
    }
    if (plan.after_nonsplit(L, kind == 1, rank, m)) {
      std::printf("end cluster %.17g %.17g %.17g %d\n", plan.reg.cr, plan.reg.ci, plan.reg.R,
                  (int)plan.reg.hp.size());
      return 0;
    }
  }
  std::printf("end open\n");
  return 0;
}
