// Executor launch shapes, written by paper_1807_02119_gb300/autotune.py from
// measurements on NVIDIA GB300 (2026-12-04 05:57 UTC); the library's defaults (pk_tuning_default).
// Batch executor, 4096 knots at q = 3, split, one launch (median ms):
//   threads  128  ktab   512     4.445
//   threads  128  ktab  1024     4.501
//   threads  128  ktab  2048     4.910
//   threads  256  ktab   512     4.269
//   threads  256  ktab  1024     4.312
//   threads  256  ktab  2048     4.308
//   threads  512  ktab   512     5.555
//   threads  512  ktab  1024     5.578
//   threads  512  ktab  2048     5.640
// Sequence runs, 192 evaluations of the scale workload, split (median ms per step):
//   outs <=  1024  work <=   4096     60.00  (6354 launches)
//   outs <=  1024  work <=  16384     60.04  (6243 launches)
//   outs <=  1024  work <=  65536     59.74  (6219 launches)
//   outs <=  2048  work <=   4096     60.22  (6352 launches)
//   outs <=  2048  work <=  16384     60.20  (6226 launches)
//   outs <=  2048  work <=  65536     60.26  (6195 launches)
//   outs <=  4096  work <=   4096     60.30  (6086 launches)
//   outs <=  4096  work <=  16384     60.28  (4362 launches)
//   outs <=  4096  work <=  65536     60.27  (4275 launches)
//   outs <=  8192  work <=   4096     59.91  (6086 launches)
//   outs <=  8192  work <=  16384     60.25  (4360 launches)
//   outs <=  8192  work <=  65536     60.31  (3898 launches)
// Tensor cores for row steps of GEMM shape from this K, split (median ms per step):
//   K >=  4     59.96
//   K >=  8     60.36
//   K >= 16     60.53
// One CTA per SM, two accumulator sets, from this many flush groups (0: never), split
// (median ms per step, measured separately after the rows above):
//   tc_db_groups =    0     56.05
//   tc_db_groups =    2     62.04
//   tc_db_groups =    3     60.23
//   tc_db_groups =    4     60.42
//   tc_db_groups =    6     60.18
// Tensor cores for row steps of GEMM shape from this many columns (tc_min_k = 4), then from
// this K (tc_min_n = 16), split (median ms per step, measured after the rows above):
//   tc_min_n =    8     54.85
//   tc_min_n =   12     54.88
//   tc_min_n =   16     54.70
//   tc_min_n =   24     54.99
//   tc_min_n =   32     56.24
//   tc_min_k =    4     55.21
//   tc_min_k =    8     53.79
//   tc_min_k =   16     53.62
// Columns again with tc_min_k = 16 (median ms per step):
//   tc_min_n =    8     53.79
//   tc_min_n =   12     53.75
//   tc_min_n =   16     54.27
//   tc_min_n =   24     53.78
//   tc_min_n =   32     56.28
// Planner cost weights (tensor-core steps: M >= 64, N >= tc_min_n, K >= tc_min_k), split
// (median ms per step, cost_gemm_milli first, then cost_out_milli with it):
//   cost_gemm_milli =   50     53.23
//   cost_gemm_milli =  100     52.60
//   cost_gemm_milli =  150     52.20
//   cost_gemm_milli =  250     53.68
//   cost_gemm_milli =  400     54.09
//   cost_out_milli  = 1000     53.95
//   cost_out_milli  = 2000     53.70
//   cost_out_milli  = 4000     52.79
//   cost_out_milli  = 8000     52.57
// After the persistent tensor-core GEMM (median ms per step, 9 replays):
//   tc_min_k = 4 / 8 / 16:            49.40 / 50.21 / 48.28
//   tc_db_groups = 0 / 2 / 3 / 4 / 6: 49.63 / 54.46 / 55.23 / 53.26 / 56.95
// Tensor cores for short-K (4 <= K < tc_min_k) row steps from this many columns:
//   tc_wide_n =  100     48.04
//   tc_wide_n =  500     48.26
//   tc_wide_n = never    50.07
//   again: 16 / 25 / 50 / 100 / never: 48.96 / 49.26 / 47.72 / 48.45 / 50.73 (50 and 100
//   differ only by a few q = 3 steps with N = 81: within run-to-run noise; 100 kept)
// Planner weights again after the persistent GEMM (median ms per step, 9 replays):
//   cost_gemm_milli = 50 / 100 / 150 / 250 / 400:  48.40 / 48.91 / 48.02 / 48.62 / 49.50
//   cost_out_milli = 1000 / 2000 / 4000 / 8000 / 16000 / 32000:
//                    49.83 / 49.91 / 48.35 / 48.64 / 48.26 / 47.74
//   cost_out_milli = 16000 / 32000 / 64000 / 128000 / 256000:
//                    49.33 / 47.89 / 48.28 / 48.97 / 48.81
// Planner cost weights again, on plans with subtree reconfiguration (frontiers of up to
// 8 subtrees), in turn: operand entry of a tensor-core step, tensor-core multiply-add,
// output entry (measured 2026-12-04 10:14 UTC; run-to-run spread about 1 ms):
// Planner: cost of a tensor-core step's operand entry (thousandths of a multiply-add), split (median ms per step):
//   cost_tcin_milli =    0     31.54
//   cost_tcin_milli =  500     31.73
//   cost_tcin_milli = 1000     32.02
//   cost_tcin_milli = 2000     32.92
//   cost_tcin_milli = 4000     29.72
//   cost_tcin_milli = 8000     36.94
//   cost_tcin_milli = 16000    412.03
// Planner: cost of a tensor-core multiply-add (thousandths of a row one), split (median ms per step):
//   cost_gemm_milli =   50     30.34
//   cost_gemm_milli =  100     29.28
//   cost_gemm_milli =  150     29.63
//   cost_gemm_milli =  250     31.96
//   cost_gemm_milli =  400     33.17
// Planner: cost of an output entry (thousandths of a multiply-add), split (median ms per step):
//   cost_out_milli = 1000     49.18
//   cost_out_milli = 2000     48.90
//   cost_out_milli = 4000     33.82
//   cost_out_milli = 8000     33.62
//   cost_out_milli = 16000     32.19
//   cost_out_milli = 32000     29.28
//   cost_out_milli = 64000     30.65
//   cost_out_milli = 128000     31.22
//   cost_out_milli = 256000     30.65
// Tensor cores for row steps again, on the reconfigured plans (16 candidates rebracketed,
// frontiers of up to 10 subtrees at the 12 largest nodes), in turn: columns, columns for
// short K, contracted extent (median ms per step, measured 2026-12-04 11:30 UTC):
//   tc_min_n =    8     28.13
//   tc_min_n =   12     28.11
//   tc_min_n =   16     28.11
//   tc_min_n =   24     28.15
//   tc_min_n =   32     34.00
//   tc_wide_n =   16     27.27
//   tc_wide_n =   25     27.17
//   tc_wide_n =   50     28.08
//   tc_wide_n =  100     28.15
//   tc_wide_n = 1073741824     31.04
//   tc_min_k =    4     27.37
//   tc_min_k =    8     27.14
//   tc_min_k =   16     27.23
// Tensor cores for row steps of GEMM shape from this many multiply-adds (median ms per
// step, 2026-12-04 11:55 UTC; 0 and 65536 tie, 65536 kept: fewer launches):
//   tc_min_work =    0     27.19
//   tc_min_work = 65536     27.19
//   tc_min_work = 262144     27.39
//   tc_min_work = 1048576     28.12
//   tc_min_work = 4194304     28.99
#pragma once
#include "pk.h"

constexpr pk_tuning kTunedDefault = {256, 512, 1024, 65536, 2048, 8, 0, 12, 100, 32000, 25, 4000, 65536};
