// Operation-counting build of the oracle (TEST INFRASTRUCTURE ONLY): the
// unchanged mfc_oracle.c compiled as C++ with every double an fc_real
// (flop_count.h), keeping its C entry points.
#include "flop_count.h"
extern "C" {
#include "mfc_oracle.c"
}
