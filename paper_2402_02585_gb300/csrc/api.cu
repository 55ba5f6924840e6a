// Status names and version of the C ABI.
#include "gqaoa.h"

extern "C" const char *gqaoa_strerror(int status) {
  switch (status) {
    case GQAOA_OK: return "ok";
    case GQAOA_EINVAL: return "invalid argument (null pointer, bad literal or misaligned buffer)";
    case GQAOA_ERANGE: return "size out of range (n, m, p, batch or shot count)";
    case GQAOA_ECUDA: return "CUDA launch or runtime error";
    case GQAOA_ETIMEOUT: return "bounded device wait gave up";
    case GQAOA_ENOMEM: return "workspace smaller than required";
    default: return "unknown status";
  }
}

extern "C" int gqaoa_version(void) { return 100; }
