// CPU harness for child_regions (cplane_strategy.h): reads a parent region,
// the split line and the two blocks' own disks; prints the children's disks.
//
// stdin:  cr ci R nhp, then nhp lines "wr wi t", then "lwr lwi lt",
//         then "c0r c0i R0" and "c1r c1i R1" (R < 0: the block is a leaf, no own disk)
// stdout: "kid cr ci R" twice
#include <cstdio>

#include "cplane_strategy.h"

int main() {
  eigdc::Region g;
  int nhp;
  if (std::scanf("%lf %lf %lf %d", &g.cr, &g.ci, &g.R, &nhp) != 4) return 2;
  for (int i = 0; i < nhp; ++i) {
    eigdc::HalfPlane h;
    if (std::scanf("%lf %lf %lf", &h.wr, &h.wi, &h.t) != 3) return 2;
    g.hp.push_back(h);
  }
  eigdc::HalfPlane L;
  if (std::scanf("%lf %lf %lf", &L.wr, &L.wi, &L.t) != 3) return 2;
  eigdc::Region own[2];
  for (int c = 0; c < 2; ++c)
    if (std::scanf("%lf %lf %lf", &own[c].cr, &own[c].ci, &own[c].R) != 3) return 2;
  eigdc::Region k0, k1;
  eigdc::child_regions(g, L, own[0].R >= 0 ? &own[0] : nullptr, own[1].R >= 0 ? &own[1] : nullptr,
                       &k0, &k1);
  std::printf("kid %.17g %.17g %.17g\nkid %.17g %.17g %.17g\n", k0.cr, k0.ci, k0.R, k1.cr, k1.ci,
              k1.R);
  return 0;
}
