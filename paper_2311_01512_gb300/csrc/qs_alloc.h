// Every device and pinned-host allocation the library makes for itself (handle
// scratch and staging ring, recorded-program arenas, circuit block matrices,
// batch tables) goes through these two calls, so that a test can make them
// fail on the host (qs_test_fail_allocations) and check that each caller
// returns QS_ERR_OOM and frees what it had taken.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

namespace qsalloc {

cudaError_t device(void** p, size_t bytes);
cudaError_t pinned(void** p, size_t bytes);

}  // namespace qsalloc
