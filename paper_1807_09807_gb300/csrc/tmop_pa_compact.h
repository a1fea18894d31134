// Software-pipelined Hessian action from the 3D FP32 compact records
// (OP_HESS_PA_C), instantiated in tmop_pa_compact.cu for the 3D (n, q) pairs
// of the element-kernel tables.
#pragma once
#include "tmop_kparams.h"

namespace tmop {

constexpr int kPacWarps = 8;  // warps (elements in flight) per block

template <int N, int Q1>
int launch_pac(const KParams& p, int grid, void* stream);
template <int N, int Q1>
int prepare_pac(int nelem, int* grid);
// the FP32 Hessian action recomputed from x through compact records built in
// shared memory (OP_HESS_C)
constexpr int kPacrWarps = 6;
template <int N, int Q1>
int launch_pacr(const KParams& p, int grid, void* stream);
template <int N, int Q1>
int prepare_pacr(int nelem, int* grid);

}  // namespace tmop
