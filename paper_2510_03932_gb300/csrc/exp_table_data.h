// Generated by gen_exp_table.py: 2^(j/32) for j = 0..31, each the double nearest the exact
// value.
static __device__ const double kExp2Table[32] = {
    0x1.0000000000000p+0,  // 0
    0x1.059b0d3158574p+0,  // 1
    0x1.0b5586cf9890fp+0,  // 2
    0x1.11301d0125b51p+0,  // 3
    0x1.172b83c7d517bp+0,  // 4
    0x1.1d4873168b9aap+0,  // 5
    0x1.2387a6e756238p+0,  // 6
    0x1.29e9df51fdee1p+0,  // 7
    0x1.306fe0a31b715p+0,  // 8
    0x1.371a7373aa9cbp+0,  // 9
    0x1.3dea64c123422p+0,  // 10
    0x1.44e086061892dp+0,  // 11
    0x1.4bfdad5362a27p+0,  // 12
    0x1.5342b569d4f82p+0,  // 13
    0x1.5ab07dd485429p+0,  // 14
    0x1.6247eb03a5585p+0,  // 15
    0x1.6a09e667f3bcdp+0,  // 16
    0x1.71f75e8ec5f74p+0,  // 17
    0x1.7a11473eb0187p+0,  // 18
    0x1.82589994cce13p+0,  // 19
    0x1.8ace5422aa0dbp+0,  // 20
    0x1.93737b0cdc5e5p+0,  // 21
    0x1.9c49182a3f090p+0,  // 22
    0x1.a5503b23e255dp+0,  // 23
    0x1.ae89f995ad3adp+0,  // 24
    0x1.b7f76f2fb5e47p+0,  // 25
    0x1.c199bdd85529cp+0,  // 26
    0x1.cb720dcef9069p+0,  // 27
    0x1.d5818dcfba487p+0,  // 28
    0x1.dfc97337b9b5fp+0,  // 29
    0x1.ea4afa2a490dap+0,  // 30
    0x1.f50765b6e4540p+0,  // 31
};
