// Host-only driver for the z-layer planner of the sweep (no GPU needed):
// reads "nz ntiles slots [preroll]" lines on stdin and prints the chosen
// plan and its modelled makespan, or "makespan ntiles slots c1 c2 ..." lines
// and prints the model's value for that plan (preroll 4).
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../paper_2404_04441_gb300/csrc/common.cuh"

int main() {
  char line[4096];
  while (std::fgets(line, sizeof line, stdin)) {
    if (std::strncmp(line, "makespan", 8) == 0) {
      long long ntiles = 0, slots = 0;
      int off = 0;
      std::sscanf(line + 8, "%lld %lld%n", &ntiles, &slots, &off);
      std::vector<int> ch;
      const char *p = line + 8 + off;
      int c, n;
      while (std::sscanf(p, "%d%n", &c, &n) == 1) {
        ch.push_back(c);
        p += n;
      }
      std::printf("%.17g\n", layer_makespan(ch, ntiles, slots));
    } else {
      int nz = 0;
      long long ntiles = 0, slots = 0;
      double pre = 4.0;
      if (std::sscanf(line, "%d %lld %lld %lf", &nz, &ntiles, &slots, &pre) < 3) continue;
      const std::vector<int> ch = plan_layers(nz, ntiles, slots, pre);
      std::printf("%.17g", layer_makespan(ch, ntiles, slots, pre));
      for (int v : ch) std::printf(" %d", v);
      std::printf("\n");
    }
  }
  return 0;
}
