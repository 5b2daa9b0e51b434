// Checkpoint / resume of a grid's state (ms_save / ms_load).  The paper has no counterpart.
//
// File layout, little-endian: the 8-byte magic "MS4CKPT1", then int32 dim, n, precision, closure,
// scheme, ncomp, the doubles z_imp and r, the int64 step, and per component its point count
// (int64) followed by the raw state: FP64 values (MS_FP64) or the FP32 hi array then the FP32 lo
// array (MS_FP32_REFINED, so a resume is bit-exact); for MS_SCHEME_C4_DE the tracked Delta E_z
// plane follows as one more component in the grid's precision.  Sources are configuration, not state: they are not
// saved.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "grid3d.cuh"
#include "k_fp64.cuh"

namespace ms {
namespace {

const char kMagic[8] = {'M', 'S', '4', 'C', 'K', 'P', 'T', '1'};

ms_status cfail(ms_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

struct Hdr {
  int dim, n, precision, closure, scheme, ncomp;
  double z_imp, r;
  long long step;
};

// Device arrays of the state (2D: E_z, H_x, H_y [+ Delta E_z]; 3D: six components).
int state_arrays(ms_grid* g, double** f64, float** hi, float** lo, size_t* n) {
  if (g->g3) return state_arrays3d(g, f64, hi, lo, n);
  for (int f = 0; f < 3; ++f) {
    f64[f] = g->f64[f];
    hi[f] = g->hi[f];
    lo[f] = g->lo[f];
    n[f] = g->sh[f].size();
  }
  if (g->de64 || g->de_hi) {
    f64[3] = g->de64;
    hi[3] = g->de_hi;
    lo[3] = g->de_lo;
    n[3] = g->sh[EZ].size();
    return 4;
  }
  return 3;
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" {

ms_status ms_save(ms_grid* g, const char* path) {
  if (!g || g->N <= 0 || !path) return cfail(MS_EINVAL, "invalid argument");
  double* f64[7];
  float* hi[7];
  float* lo[7];
  size_t n[7];
  const int nc = state_arrays(g, f64, hi, lo, n);
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) return cfail(MS_ECUDA, "stream synchronisation failed");
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return cfail(MS_EINVAL, std::string("cannot open ") + path + " for writing");
  Hdr h{g->desc.dim, g->desc.n, g->desc.precision, g->desc.closure, g->desc.scheme, nc, g->desc.z_imp, g->desc.r,
        (long long)g->step};
  bool ok = std::fwrite(kMagic, 1, 8, fp) == 8;
  const int ints[6] = {h.dim, h.n, h.precision, h.closure, h.scheme, h.ncomp};
  ok = ok && std::fwrite(ints, sizeof(int), 6, fp) == 6;
  ok = ok && std::fwrite(&h.z_imp, sizeof(double), 1, fp) == 1 && std::fwrite(&h.r, sizeof(double), 1, fp) == 1;
  ok = ok && std::fwrite(&h.step, sizeof(long long), 1, fp) == 1;
  for (int c = 0; c < nc && ok; ++c) {
    const long long cnt = (long long)n[c];
    ok = std::fwrite(&cnt, sizeof(long long), 1, fp) == 1;
    if (f64[c]) {
      std::vector<double> buf(n[c]);
      ok = ok && cudaMemcpy(buf.data(), f64[c], n[c] * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
      ok = ok && std::fwrite(buf.data(), sizeof(double), n[c], fp) == n[c];
    } else {
      std::vector<float> buf(n[c]);
      for (float* arr : {hi[c], lo[c]}) {
        ok = ok && cudaMemcpy(buf.data(), arr, n[c] * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess;
        ok = ok && std::fwrite(buf.data(), sizeof(float), n[c], fp) == n[c];
      }
    }
  }
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? MS_OK : cfail(MS_ECUDA, std::string("writing checkpoint ") + path + " failed");
}

ms_status ms_load(ms_grid* g, const char* path) {
  if (!g || g->N <= 0 || !path) return cfail(MS_EINVAL, "invalid argument");
  double* f64[7];
  float* hi[7];
  float* lo[7];
  size_t n[7];
  const int nc = state_arrays(g, f64, hi, lo, n);
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return cfail(MS_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int ints[6];
  Hdr h{};
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kMagic, 8) == 0;
  ok = ok && std::fread(ints, sizeof(int), 6, fp) == 6;
  ok = ok && std::fread(&h.z_imp, sizeof(double), 1, fp) == 1 && std::fread(&h.r, sizeof(double), 1, fp) == 1;
  ok = ok && std::fread(&h.step, sizeof(long long), 1, fp) == 1;
  if (!ok) {
    std::fclose(fp);
    return cfail(MS_EINVAL, std::string(path) + " is not a checkpoint of this library");
  }
  if (ints[0] != g->desc.dim || ints[1] != g->desc.n || ints[2] != g->desc.precision || ints[3] != g->desc.closure ||
      ints[4] != g->desc.scheme || ints[5] != nc || h.z_imp != g->desc.z_imp || h.r != g->desc.r) {
    std::fclose(fp);
    return cfail(MS_EINVAL, "checkpoint descriptor (dim, n, precision, closure, scheme, z_imp, r) differs from the grid's");
  }
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
    std::fclose(fp);
    return cfail(MS_ECUDA, "stream synchronisation failed");
  }
  // the whole payload is read and checked on the host first: a truncated or inconsistent file
  // leaves the grid's state untouched
  std::vector<std::vector<double>> b64(nc);
  std::vector<std::vector<float>> b32(2 * nc);
  for (int c = 0; c < nc && ok; ++c) {
    long long cnt = 0;
    ok = std::fread(&cnt, sizeof(long long), 1, fp) == 1 && cnt == (long long)n[c];
    if (!ok) break;
    if (f64[c]) {
      b64[c].resize(n[c]);
      ok = std::fread(b64[c].data(), sizeof(double), n[c], fp) == n[c];
    } else {
      for (int part = 0; part < 2 && ok; ++part) {
        b32[2 * c + part].resize(n[c]);
        ok = std::fread(b32[2 * c + part].data(), sizeof(float), n[c], fp) == n[c];
      }
    }
  }
  if (ok) {  // nothing may follow the last component
    char extra;
    ok = std::fread(&extra, 1, 1, fp) == 0;
  }
  std::fclose(fp);
  if (!ok) return cfail(MS_EINVAL, std::string("checkpoint ") + path + " is truncated or inconsistent");
  for (int c = 0; c < nc; ++c) {
    bool cp;
    if (f64[c]) {
      cp = cudaMemcpy(f64[c], b64[c].data(), n[c] * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
    } else {
      cp = cudaMemcpy(hi[c], b32[2 * c].data(), n[c] * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(lo[c], b32[2 * c + 1].data(), n[c] * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!cp) return cfail(MS_ECUDA, "copying the checkpoint to the device failed");
  }
  g->step = (long)h.step;
  if (g->d_step && cudaMemcpy(g->d_step, &g->step, sizeof(long), cudaMemcpyHostToDevice) != cudaSuccess)
    return cfail(MS_ECUDA, "restoring the device step index failed");
  return MS_OK;
}

}  // extern "C"
