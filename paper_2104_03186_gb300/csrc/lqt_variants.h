// (scalar type, state size n, control size m) combinations compiled into the
// library.  Each list is expanded by the instantiation units and by the
// dispatch table of the C ABI.
#pragma once

#define LQT_VARIANTS_F32_SMALL(X) X(float, 1, 1) X(float, 2, 1) X(float, 2, 2) X(float, 3, 1) X(float, 3, 2)
#define LQT_VARIANTS_F32_N4(X) X(float, 4, 1) X(float, 4, 2) X(float, 4, 4)
#define LQT_VARIANTS_F64(X) X(double, 1, 1) X(double, 2, 1) X(double, 4, 2)

#define LQT_VARIANTS(X) LQT_VARIANTS_F32_SMALL(X) LQT_VARIANTS_F32_N4(X) LQT_VARIANTS_F64(X)
