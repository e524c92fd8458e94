// Executor launch shapes, written by paper_1807_02119_gb300/autotune.py from
// measurements on NVIDIA GB300 (2026-12-04 05:08 UTC); the library's defaults (pk_tuning_default).
// Batch executor, 4096 knots at q = 3, split, one launch (median ms):
//   threads  128  ktab   512     4.585
//   threads  128  ktab  1024     4.541
//   threads  128  ktab  2048     4.956
//   threads  256  ktab   512     4.243
//   threads  256  ktab  1024     4.278
//   threads  256  ktab  2048     4.292
//   threads  512  ktab   512     5.530
//   threads  512  ktab  1024     5.580
//   threads  512  ktab  2048     5.683
// Sequence runs, 192 evaluations of the scale workload, split (median ms per step):
//   outs <=  1024  work <=   4096     68.08  (6471 launches)
//   outs <=  1024  work <=  16384     67.58  (6360 launches)
//   outs <=  1024  work <=  65536     67.39  (6336 launches)
//   outs <=  2048  work <=   4096     67.68  (6469 launches)
//   outs <=  2048  work <=  16384     68.12  (6343 launches)
//   outs <=  2048  work <=  65536     67.82  (6312 launches)
//   outs <=  4096  work <=   4096     68.11  (6203 launches)
//   outs <=  4096  work <=  16384     68.13  (4479 launches)
//   outs <=  4096  work <=  65536     67.69  (4392 launches)
//   outs <=  8192  work <=   4096     69.44  (6203 launches)
//   outs <=  8192  work <=  16384     67.96  (4477 launches)
//   outs <=  8192  work <=  65536     69.28  (4015 launches)
#pragma once
#include "pk.h"

constexpr pk_tuning kTunedDefault = {256, 512, 1024, 65536, 2048};
