// capi_types.cuh -- the opaque handle types behind include/gwhe.h, shared by
// the translation units that implement the C ABI.
#pragma once

#include "../../include/gwhe.h"
#include "gwas.cuh"

struct gwhe_ctx {
  gwhe::Context* c;
};
struct gwhe_ct {
  gwhe_ctx* owner;
  gwhe::CtPtr ct;
};
struct gwhe_job {
  gwhe_ctx* owner;
  std::unique_ptr<gwhe::Job> job;
};
