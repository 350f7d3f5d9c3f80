// Generated kernels for thin tail segments (codegen.cu).
#pragma once

#include <string>

#include "plan.cuh"
#include "tail.cuh"

namespace sptrsv {

// Largest segment (rows) a kernel is generated for: its unknowns sit in one
// CTA's shared memory (8 B each), and compiling takes ~1.3 ms per row.
constexpr int32_t kCodegenMaxRows = 4096;

// The view of a segment the tail kernels take (tail.cu).
TailData tail_view(const TailSeg &t);

// Whether segment sg may get a generated kernel under the caller's limit.
bool codegen_eligible(const TailSeg &sg, int32_t max_rows);
// The source of a segment's kernel from host copies of its records (the
// layout of TailData): empty with thin = false when a kernel would not pay
// (some level is not thin enough, or a term reads x beyond the window).
sptrsv_status_t source_from_records(int32_t nr, int32_t K, int32_t nlev, const int32_t *row,
                                    const int32_t *nn, const int4 *term, const double2 *dg,
                                    std::string &src, bool &thin);
// The same for segment sg (its records copied from the device).
sptrsv_status_t codegen_source(const TailSeg &sg, std::string &src, bool &thin);
// Generates, compiles and loads sg's kernel into sg.gen (left empty when the
// segment is not thin); ms accumulates the time taken.  SPTRSV_ERR_CODEGEN
// when the runtime compiler is missing or rejects the source.
sptrsv_status_t codegen_build(TailSeg &sg, double &ms);
// The fold pass of the segment, then its generated kernel (one thread).
cudaError_t codegen_launch(const TailSeg &sg, const double *b, double *x, cudaStream_t s);
// Name of the generated kernel's entry point.
const char *codegen_entry_name();

}  // namespace sptrsv
