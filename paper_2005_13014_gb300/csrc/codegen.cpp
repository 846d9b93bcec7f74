// codegen.cpp - generic stencil programs (no hand-written kernel).
#include "../../include/oec.h"
#include "api_internal.h"

struct oec_generic_state {};

namespace oec {

bool generic_schedule_ok(const oec_schedule& s, std::string& why) {
  if (s.fusion != OEC_FUSE_INLINE && s.fusion != OEC_FUSE_NONE) { why = "unknown fusion"; return false; }
  return true;
}

void generic_release(oec_program* p) {
  delete p->gen;
  p->gen = nullptr;
}

int generic_apply(oec_program*, const oec_field_desc*, const oec_field_desc*, const int64_t*, const int64_t*,
                  const double*, cudaStream_t) {
  return fail(OEC_ERR_UNSUPPORTED, "this program has no hand-written kernel and the generic generator is not built");
}

}  // namespace oec
