// The library's double-float arithmetic (pd_df.cuh) compiled as host C++,
// driven in the order the S products use it: entry p of a row segment goes
// to lane p mod 32 and, while four more strides of 32 remain, to accumulator
// (p / 32) mod 4 of that lane (else accumulator 0); each lane adds its four
// accumulators pairwise, and the lanes are combined by the xor butterfly of a
// warp-wide sum (emulated here lane by lane with df_add).
#define __device__
#define __forceinline__ inline
#include "../../paper_2605_14526_b300/csrc/pd_df.cuh"

using namespace pdk;

extern "C" {
// out: [32][2] (hi, lo) of every lane after the butterfly
void df_segment_dot(int n, const double* s, const double* x, float* out) {
  float ah[32][4], al[32][4];
  for (int l = 0; l < 32; ++l)
    for (int u = 0; u < 4; ++u) ah[l][u] = al[l][u] = 0.0f;
  for (int l = 0; l < 32; ++l) {
    int p = l;
    for (; p + 96 < n; p += 128)
      for (int u = 0; u < 4; ++u) df_mac(ah[l][u], al[l][u], df_split(s[p + 32 * u]), df_split(x[p + 32 * u]));
    for (; p < n; p += 32) df_mac(ah[l][0], al[l][0], df_split(s[p]), df_split(x[p]));
  }
  float2 v[32], w[32];
  for (int l = 0; l < 32; ++l)
    v[l] = df_add(df_add(make_float2(ah[l][0], al[l][0]), make_float2(ah[l][1], al[l][1])),
                  df_add(make_float2(ah[l][2], al[l][2]), make_float2(ah[l][3], al[l][3])));
  for (int o = 16; o > 0; o >>= 1) {
    for (int l = 0; l < 32; ++l) w[l] = df_add(v[l], v[l ^ o]);
    for (int l = 0; l < 32; ++l) v[l] = w[l];
  }
  for (int l = 0; l < 32; ++l) {
    out[2 * l] = v[l].x;
    out[2 * l + 1] = v[l].y;
  }
}

void df_split_join(int n, const double* x, float* hl, double* back) {
  for (int i = 0; i < n; ++i) {
    const float2 a = df_split(x[i]);
    hl[2 * i] = a.x;
    hl[2 * i + 1] = a.y;
    back[i] = df_join(a);
  }
}
}
