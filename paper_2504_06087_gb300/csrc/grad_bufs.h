// Scratch buffers of the parameter-gradient call, carved from one workspace
// region.  The same routine sizes the region (base == nullptr) and assigns
// the pointers, so the plan and the pipeline agree by construction.
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace fire {

template <typename T>
struct GradBufs {
  T *HL, *ZL;                          // [L+1][nb][d], [L][nb][d]
  T *JZ1[2], *JA1[2], *JZ2[2], *JA2[2];  // [nb][J]
  T *SU;                               // [nb][R + RD]
  T *VZ1[2], *VA1[2], *VZ2[2], *VA2[2];  // [Wc][J]
  T *dO, *dF;                          // [nb][D n]
  T *dH, *dZ, *dH0, *dP5, *dY5, *dS5, *dyx;  // [nb][d]
  T *dQf;                              // [nb][N E]
  T *df, *dY2, *dZ2, *dA1, *dZ1;       // [nb], [nb][J] x 4
  T *dV, *dfv, *dVY2, *dVZ2, *dVA1, *dVZ1;   // [Wc][RD], [Wc], [Wc][J] x 4
  T *dSU;                              // [nb][R + RD]
  T *dPm, *dQm;                        // [nb][2d]
  T *dZ5;                              // [nb][2d]
  T *AT;                               // [Wc][D][n][n]
  float *Phif;                         // [Wc][D][n][n]

  static size_t carve(void* base, GradBufs* g, int64_t Wc, int n, int d, int L, int D, int J, int R, int RD,
                      int NE) {
    size_t o = 0;
    unsigned char* b = reinterpret_cast<unsigned char*>(base);
    auto take = [&](int64_t count, size_t es) -> void* {
      size_t r = o;
      o = (o + (size_t)count * es + 255) & ~(size_t)255;
      return b ? b + r : nullptr;
    };
    const int64_t nb = Wc * n, Dn = (int64_t)D * n;
    GradBufs tmp;
    GradBufs* q = g ? g : &tmp;
    q->HL = (T*)take((L + 1) * nb * d, sizeof(T));
    q->ZL = (T*)take((L > 0 ? L : 1) * nb * d, sizeof(T));
    for (int k = 0; k < 2; ++k) {
      q->JZ1[k] = (T*)take(nb * J, sizeof(T));
      q->JA1[k] = (T*)take(nb * J, sizeof(T));
      q->JZ2[k] = (T*)take(nb * J, sizeof(T));
      q->JA2[k] = (T*)take(nb * J, sizeof(T));
      q->VZ1[k] = (T*)take(Wc * J, sizeof(T));
      q->VA1[k] = (T*)take(Wc * J, sizeof(T));
      q->VZ2[k] = (T*)take(Wc * J, sizeof(T));
      q->VA2[k] = (T*)take(Wc * J, sizeof(T));
    }
    q->SU = (T*)take(nb * (R + RD), sizeof(T));
    q->dO = (T*)take(nb * Dn, sizeof(T));
    q->dF = (T*)take(nb * Dn, sizeof(T));
    q->dH = (T*)take(nb * d, sizeof(T));
    q->dZ = (T*)take(nb * d, sizeof(T));
    q->dH0 = (T*)take(nb * d, sizeof(T));
    q->dP5 = (T*)take(nb * d, sizeof(T));
    q->dY5 = (T*)take(nb * d, sizeof(T));
    q->dS5 = (T*)take(nb * d, sizeof(T));
    q->dyx = (T*)take(nb * d, sizeof(T));
    q->dQf = (T*)take(nb * NE, sizeof(T));
    q->df = (T*)take(nb, sizeof(T));
    q->dY2 = (T*)take(nb * J, sizeof(T));
    q->dZ2 = (T*)take(nb * J, sizeof(T));
    q->dA1 = (T*)take(nb * J, sizeof(T));
    q->dZ1 = (T*)take(nb * J, sizeof(T));
    q->dV = (T*)take(Wc * RD, sizeof(T));
    q->dfv = (T*)take(Wc, sizeof(T));
    q->dVY2 = (T*)take(Wc * J, sizeof(T));
    q->dVZ2 = (T*)take(Wc * J, sizeof(T));
    q->dVA1 = (T*)take(Wc * J, sizeof(T));
    q->dVZ1 = (T*)take(Wc * J, sizeof(T));
    q->dSU = (T*)take(nb * (R + RD), sizeof(T));
    q->dPm = (T*)take(nb * 2 * d, sizeof(T));
    q->dQm = (T*)take(nb * 2 * d, sizeof(T));
    q->dZ5 = (T*)take(nb * 2 * d, sizeof(T));
    q->AT = (T*)take(Wc * D * (int64_t)n * n, sizeof(T));
    q->Phif = (float*)take(Wc * D * (int64_t)n * n, sizeof(float));
    return o;
  }
};

}  // namespace fire
