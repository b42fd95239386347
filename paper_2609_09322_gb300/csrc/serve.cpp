// serve.cpp -- continuous-batching request server (placeholder until built).
#include "runtime.h"

namespace gbd {

void serve_shutdown(Ctx &) {}

}  // namespace gbd
