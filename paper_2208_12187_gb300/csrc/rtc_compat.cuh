// The few standard-library names the device headers use.  Under nvcc they
// come from the usual headers; under NVRTC (user-defined models are compiled
// at run time from these same headers) there is no host standard library, so
// they are declared here.
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
#ifndef INFINITY
#define INFINITY (__int_as_float(0x7f800000))
#endif
namespace std {
template <class A, class B> struct is_same { static constexpr bool value = false; };
template <class A> struct is_same<A, A> { static constexpr bool value = true; };
}  // namespace std
#else
#include <cstddef>
#include <cstdint>
#include <cmath>
#include <type_traits>
#include <cuda_runtime.h>
#endif
