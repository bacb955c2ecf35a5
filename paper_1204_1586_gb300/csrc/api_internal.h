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

// The argument status cp_gradient_all returns for these arguments (shape,
// precision, split and pointer checks, in its order), CPG_OK when they are
// valid; it launches nothing.
cpg_status gradient_all_arg_status(const void* Y, const int64_t* I, int N, const void* const* A, int R,
                                   void* const* G, const cpg_opts* opts);

// Bytes of workspace cp_gradient_all needs given opts->workspace_bytes of
// room: those of the plan it would run (the measured plan when that fits,
// else the planner's), less the optional pitched copy of Y.  0 on invalid
// arguments.
size_t gradient_all_bytes_for(const int64_t* I, int N, int R, const cpg_opts* opts);

}  // namespace cpg
