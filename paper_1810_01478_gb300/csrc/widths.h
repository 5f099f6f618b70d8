// Limb counts per lane (M = n/32, bits = 1024 M) compiled into libhk.
// The build compiles inst.cu once per entry with -DHK_M=<M>.
#pragma once
#define HK_FOR_EACH_M(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(12) X(16) X(24)
