// Compile-time pass list of the fast FFT family (Stockham autosort) and the
// layout of its twiddle table.  P = R_0 * R_1 * ... with R_i = min(MR, what
// is left): MR = 16 gives 16,16,.. then the remainder; MR = 32 likewise.
// Used by the table generator (plan.cu) and by the kernels, so both agree.
#pragma once

namespace pfb {

constexpr int fft_npasses(int P, int MR) {
    int n = 0, rem = P;
    while (rem > 1) { rem /= (rem < MR ? rem : MR); ++n; }
    return n;
}

// radix of pass i
constexpr int fft_radix(int P, int i, int MR) {
    int rem = P;
    for (int k = 0; k < i; ++k) rem /= (rem < MR ? rem : MR);
    return rem < MR ? rem : MR;
}

// Ns (product of the radices before pass i)
constexpr int fft_ns(int P, int i, int MR) {
    int ns = 1;
    for (int k = 0; k < i; ++k) ns *= fft_radix(P, k, MR);
    return ns;
}

// offset of pass i's entries in the twiddle table (passes with Ns > 1 only):
// entries [(j mod Ns)*(R-1) + r-1] = exp(-2 pi i r (j mod Ns) / (Ns R))
constexpr int fft_tw_offset(int P, int i, int MR) {
    int off = 0;
    for (int k = 0; k < i; ++k) {
        int ns = fft_ns(P, k, MR);
        if (ns > 1) off += ns * (fft_radix(P, k, MR) - 1);
    }
    return off;
}

constexpr int fft_tw_entries(int P, int MR) { return fft_tw_offset(P, fft_npasses(P, MR), MR); }

}  // namespace pfb
