// Host check of the range checks of the checked build (csrc/tsdf_check.h):
// in-range indices pass and leave the error word alone; out-of-range ones
// (past the end, negative, far past) fail and set exactly the BOUNDS bit; a
// null error word is tolerated. Built without TSDF_CHECKED, every index
// passes and nothing is recorded. Prints "ok" when every case holds.
#include <cstdio>

#include "tsdf_check.h"

static int failures = 0;

static void expect(bool cond, const char* what) {
  if (!cond) {
    std::printf("FAILED: %s\n", what);
    ++failures;
  }
}

int main() {
  unsigned int err = 0;
  const unsigned long long n = 1000;
  expect(tsdf::index_ok(0, n, &err), "first index in range");
  expect(tsdf::index_ok(n - 1, n, &err), "last index in range");
  expect(err == 0, "in-range indices leave the error word alone");
  expect(tsdf::index_ok_signed(0, n, &err) && tsdf::index_ok_signed(999, n, &err),
         "signed indices in range");
  expect(err == 0, "in-range signed indices leave the error word alone");
#ifdef TSDF_CHECKED
  expect(!tsdf::index_ok(n, n, &err), "one past the end fails");
  expect(err == TSDF_ERRBIT_BOUNDS, "the BOUNDS bit alone is set");
  err = TSDF_ERRBIT_POOL_FULL;
  expect(!tsdf::index_ok(1ull << 40, n, &err), "far past the end fails");
  expect(err == (TSDF_ERRBIT_POOL_FULL | TSDF_ERRBIT_BOUNDS), "other bits are kept");
  err = 0;
  expect(!tsdf::index_ok_signed(-1, n, &err), "a negative index fails");
  expect(!tsdf::index_ok_signed(static_cast<long long>(n), n, &err), "signed one past the end fails");
  expect(err == TSDF_ERRBIT_BOUNDS, "signed failures set the BOUNDS bit");
  expect(!tsdf::index_ok(0, 0, nullptr), "an empty range fails, with no error word");
#else
  expect(tsdf::index_ok(n, n, &err) && tsdf::index_ok_signed(-1, n, &err),
         "unchecked builds pass every index");
  expect(err == 0, "unchecked builds record nothing");
#endif
  if (failures == 0) std::printf("ok\n");
  return failures == 0 ? 0 : 1;
}
