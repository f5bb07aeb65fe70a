// Two FP32 lanes per instruction: the packed add/sub/mul/fma of sm_100 and
// later on .b64 register pairs, each lane rounded to nearest exactly as the
// scalar FP32 instruction would round it.
#pragma once

namespace tri {

using f2 = unsigned long long;

__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
#define TRI_F2_OP(NAME, OP)                                                                                   \
    __device__ __forceinline__ f2 NAME(f2 a, f2 b)                                                           \
    {                                                                                                        \
        f2 r;                                                                                                \
        asm(OP ".rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));                                          \
        return r;                                                                                            \
    }
TRI_F2_OP(f2_add, "add")
TRI_F2_OP(f2_sub, "sub")
TRI_F2_OP(f2_mul, "mul")
#undef TRI_F2_OP
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

}  // namespace tri
