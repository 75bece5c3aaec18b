// swe_batch.h -- host-side interface of the persistent batch kernel
// (declared with the other launchers in swe_launch.h).
#pragma once
#include "swe_launch.h"
