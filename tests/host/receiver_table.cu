// Host-only driver for the receiver table of the sweep (no GPU needed).
// stdin: "nx ny nz tx ty nrec" then nrec lines "x y z". stdout: the status,
// then one line "z local id tile" per entry, then the ntiles + 1 starts.
#include <cstdio>
#include <vector>

#include "../../paper_2404_04441_gb300/csrc/common.cuh"

int main() {
  int nx, ny, nz, tx, ty, nrec;
  if (std::scanf("%d %d %d %d %d %d", &nx, &ny, &nz, &tx, &ty, &nrec) != 6) return 2;
  std::vector<int32_t> xyz((size_t)nrec * 3);
  for (int i = 0; i < 3 * nrec; ++i)
    if (std::scanf("%d", &xyz[i]) != 1) return 2;
  const int ntx = (nx + tx - 1) / tx, nty = (ny + ty - 1) / ty;
  std::vector<int4> entries;
  std::vector<int> start;
  const int st = build_receiver_table(xyz.data(), nrec, nx, ny, nz, tx, ty, ntx,
                                      ntx * nty, entries, start);
  std::printf("%d\n", st);
  if (st != WAVE_OK) return 0;
  for (const int4 &e : entries) std::printf("%d %d %d %d\n", e.x, e.y, e.z, e.w);
  for (int v : start) std::printf("%d\n", v);
  return 0;
}
