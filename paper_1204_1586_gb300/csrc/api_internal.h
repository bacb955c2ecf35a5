// Library-internal entry points shared between translation units (not part of
// the C ABI of include/cpgrad.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/cpgrad.h"

namespace cpg {

// Bytes of workspace `call` cannot run without: cpg_workspace_size less the
// optional pitched copy of Y (a call given less room for the copy streams Y
// itself).
size_t workspace_bytes_required(const int64_t* I, int N, int R, const cpg_opts* opts, int call);

}  // namespace cpg
