// hq_fault.cuh -- injected failures of the library's scratch allocations
// (tests of the error paths; see hq_test_fail_next_allocs in hq.h).
#pragma once

namespace hq {

// true (and one fewer injected failure left) when the caller's scratch
// allocation is to fail as if the device were out of memory
bool injected_alloc_failure();

}  // namespace hq
