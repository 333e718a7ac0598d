// Host-side check of the candidate key encoding used by the kernels: order
// preservation of FP32 scores, folding of -0.0, id tie-break, round trip.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "lr_internal.h"

int main() {
  using namespace lr;
  std::vector<float> v = {-INFINITY, -3.5f, -1.0f, -1e-30f, -0.0f, 0.0f, 1e-38f, 1e-30f, 0.25f, 1.0f, 3.5f, INFINITY};
  int bad = 0;
  for (size_t i = 0; i + 1 < v.size(); ++i) {
    uint32_t a = score_key(v[i]), b = score_key(v[i + 1]);
    bool eq = (v[i] == v[i + 1]);
    if (eq ? a != b : !(a < b)) { std::printf("order fails at %zu\n", i); ++bad; }
  }
  for (float f : v) {
    float r = key_score(score_key(f));
    if (!(r == f) && !(std::isinf(f) && r == f)) { std::printf("round trip fails for %g\n", f); ++bad; }
  }
  // equal scores: the smaller id gets the larger key
  if (!(make_key(0.5f, 3) > make_key(0.5f, 7))) { std::printf("id tie-break fails\n"); ++bad; }
  if (!(make_key(0.6f, 7) > make_key(0.5f, 3))) { std::printf("score dominance fails\n"); ++bad; }
  if (key_id(make_key(-2.0f, 123456789u)) != 123456789u) { std::printf("id round trip fails\n"); ++bad; }
  if (make_key(-0.0f, 5) != make_key(0.0f, 5)) { std::printf("-0.0 not folded\n"); ++bad; }
  std::srand(7);
  for (int t = 0; t < 100000; ++t) {
    float a = (float)(std::rand() - RAND_MAX / 2) / 1e6f, b = (float)(std::rand() - RAND_MAX / 2) / 1e6f;
    if ((a < b) != (score_key(a) < score_key(b))) { ++bad; break; }
  }
  std::printf(bad ? "FAIL\n" : "OK\n");
  return bad ? 1 : 0;
}
