// schemes.cuh -- the two test equations of Section 4.2: heat.cuh (FTCS) and
// euler.cuh (second-order finite volume, pressure-ratio minmod limiter).
#pragma once
#include "euler.cuh"
#include "heat.cuh"
#include "heat_policy.cuh"
