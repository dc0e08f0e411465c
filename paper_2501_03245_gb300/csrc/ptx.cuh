// PTX carry-chain primitives for multi-precision integer arithmetic.
//
// Each wrapper is one PTX instruction.  Consecutive calls form a carry chain
// through the condition-code register CC: a chain starts with a non-"c"
// instruction (add.cc / mad.lo.cc) and continues with the "c" forms
// (addc.cc / madc.*.cc).  Callers keep chains contiguous: nothing that writes CC
// may be placed between two links of a chain.  The asm statements are volatile
// so the front end keeps their order; ptxas tracks CC as a real dependency.
//
// The multiply-add pairs mad.lo.cc / madc.hi.cc on the same operands are the
// "mad_n" building block of Section 4.1 (the paper's Table 2 maps the pair to
// one IMAD.WIDE.X issue).
#pragma once
#include <cstdint>

#ifndef ECC_DEV
#define ECC_DEV __device__ __forceinline__
#endif

namespace ptx {

ECC_DEV uint32_t add_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
ECC_DEV uint32_t addc_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
ECC_DEV uint32_t addc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("addc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
ECC_DEV uint32_t sub_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
ECC_DEV uint32_t subc_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
ECC_DEV uint32_t subc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("subc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
// lo(a*b) + c, starting a chain
ECC_DEV uint32_t mad_lo_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("mad.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
ECC_DEV uint32_t madc_lo_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("madc.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
ECC_DEV uint32_t mad_hi_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("mad.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
ECC_DEV uint32_t madc_hi_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("madc.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
ECC_DEV uint32_t madc_hi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("madc.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// Asynchronous 16-byte global -> shared copies (cp.async, cached in L2 only):
// the data lands in shared memory without passing through registers, so a
// thread can fetch its next item's operands while it computes on the current
// one.  A thread reads back only what it copied itself, after wait_all.
ECC_DEV void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
ECC_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
ECC_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// all but the most recently committed group
ECC_DEV void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

}  // namespace ptx
