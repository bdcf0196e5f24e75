// Compile-time pass list of the fast FFT family (Stockham autosort, radix 16
// first, one final radix in {2, 4, 8, 16}) and the layout of its twiddle table.
// Used by the table generator (plan.cu) and by the kernels, so both agree.
#pragma once

namespace pfb {

constexpr int fft_npasses(int P) {
    int n = 0, rem = P;
    while (rem >= 256 || rem == 16) { ++n; rem /= 16; }
    if (rem > 16) { ++n; rem /= 16; }
    if (rem > 1) ++n;
    return n;
}

// radix of pass i
constexpr int fft_radix(int P, int i) {
    int rem = P, k = 0;
    while (rem >= 256 || rem == 16) { if (k == i) return 16; ++k; rem /= 16; }
    if (rem > 16) { if (k == i) return 16; ++k; rem /= 16; }
    if (rem > 1 && k == i) return rem;
    return 1;
}

// Ns (product of the radices before pass i)
constexpr int fft_ns(int P, int i) {
    int ns = 1;
    for (int k = 0; k < i; ++k) ns *= fft_radix(P, k);
    return ns;
}

// offset of pass i's entries in the twiddle table (passes with Ns > 1 only)
constexpr int fft_tw_offset(int P, int i) {
    int off = 0;
    for (int k = 0; k < i; ++k) {
        int ns = fft_ns(P, k);
        if (ns > 1) off += ns * (fft_radix(P, k) - 1);
    }
    return off;
}

constexpr int fft_tw_entries(int P) { return fft_tw_offset(P, fft_npasses(P)); }

}  // namespace pfb
