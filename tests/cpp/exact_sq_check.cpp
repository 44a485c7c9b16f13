// Host check of tqs::sq_f32_as_f64_bits against the FPU: every exponent,
// subnormals, zeros, both signs, and random bit patterns.
#include "exact_sq.h"
#include <cstdio>
#include <cstring>
#include <random>
#include <cmath>
#include <limits>
int main(){
  std::mt19937_64 g(1);
  long bad=0, n=0;
  auto check=[&](uint32_t bits){
    float x; std::memcpy(&x,&bits,4);
    if(!std::isfinite(x)) return;
    double want=(double)x*(double)x; uint64_t wb; std::memcpy(&wb,&want,8);
    uint64_t got=tqs::sq_f32_as_f64_bits(bits);
    n++; if(got!=wb){ if(bad<5) printf("mismatch %08x %a got %016llx want %016llx\n",bits,x,(unsigned long long)got,(unsigned long long)wb); bad++;}
  };
  for(uint32_t e=0;e<255;e++) for(uint32_t k=0;k<2000;k++){ uint32_t m=(k<4)? (k==0?0:(k==1?1:(k==2?0x7fffff:0x400000))) : (uint32_t)(g()&0x7fffff); check((e<<23)|m); check(0x80000000u|(e<<23)|m);}
  for(long i=0;i<3000000;i++) check((uint32_t)g());
  printf("checked %ld, mismatches %ld\n",n,bad); return bad!=0;
}
