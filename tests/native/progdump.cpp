// progdump.cpp -- test helper: runs the library's host-side mechanism compiler
// (csrc/mechanism.cpp, no GPU needed) on a reaction table and writes the
// per-cell layout, the pivot order, the symbolic fill and every warp program
// as text, so that tests can replay the programs on the CPU.
//
// usage: progdump <in.bin> <out.txt>; in.bin = int32 n_species, int32
// n_reactions, then n_reactions chem_reaction records.
#include <cstdio>
#include <vector>

#include "internal.h"

using namespace chemgpu;

// the constant-memory upload lives with the kernels; the compiler only calls it
namespace chemgpu {
cudaError_t set_constants() { return cudaSuccess; }
}

static void dump_prog(FILE *f, const char *name, const HostProgram &p) {
  std::fprintf(f, "%s %d\n", name, p.n_pass());
  for (const Op &o : p.ops) std::fprintf(f, "%u %u %u %u\n", o.t, o.a, o.b, o.c);
  std::fprintf(f, "units_%s", name);
  for (uint8_t u : p.unit) std::fprintf(f, " %d", (int)u);
  std::fprintf(f, "\n");
}

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *in = std::fopen(argv[1], "rb");
  if (!in) return 3;
  int S = 0, R = 0;
  if (std::fread(&S, 4, 1, in) != 1 || std::fread(&R, 4, 1, in) != 1) return 4;
  std::vector<chem_reaction> rx(R > 0 ? R : 1);
  if (R > 0 && std::fread(rx.data(), sizeof(chem_reaction), R, in) != (size_t)R) return 5;
  std::fclose(in);
  Mechanism m;
  std::string msg;
  if (int rc = compile_mechanism(S, R, rx.data(), m, msg)) {
    std::printf("compile failed %d %s\n", rc, msg.c_str());
    return 1;
  }
  FILE *f = std::fopen(argv[2], "w");
  if (!f) return 6;
  const MechDev &d = m.dev;
  std::fprintf(f, "layout %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", d.Wd_len, d.d_Y, d.d_KT, d.d_RT, d.d_F, d.d_ONE,
               d.d_ZERO, d.WL_len, d.L_LU, d.L_X, d.L_P, d.L_ZERO, d.nnz_lu, d.m_clear);
  std::fprintf(f, "adj %d %d %d %d %d %d\n", d.Wda_len, d.a_MU, d.a_NM, d.a_PP, d.a_JTM, d.a_G);
  std::fprintf(f, "pos");
  for (int v : m.pos) std::fprintf(f, " %d", v);
  std::fprintf(f, "\nludiag");
  for (int v : m.lu_diag) std::fprintf(f, " %d", v);
  std::fprintf(f, "\npairrx");
  for (int v : m.pair_rx) std::fprintf(f, " %d", v);
  std::fprintf(f, "\npairother");
  for (auto &v : m.pair_other) std::fprintf(f, " %d %d", v.first, v.second);
  std::fprintf(f, "\ndconst");
  for (size_t i = 0; i < m.d_consts_v.size(); ++i) std::fprintf(f, " %d %.17g", m.d_consts_i[i], m.d_consts_v[i]);
  std::fprintf(f, "\nLconst");
  for (size_t i = 0; i < m.L_consts_v.size(); ++i) std::fprintf(f, " %d %.17g", m.L_consts_i[i], m.L_consts_v[i]);
  std::fprintf(f, "\naconst");
  for (size_t i = 0; i < m.a_consts_v.size(); ++i) std::fprintf(f, " %d %.17g", m.a_consts_i[i], m.a_consts_v[i]);
  std::fprintf(f, "\nfill");
  for (uint8_t v : m.fill) std::fprintf(f, " %d", (int)v);
  std::fprintf(f, "\ninfo %d %d\n", m.nnz_jac, m.nnz_lu);
  dump_prog(f, "f", m.f_prog);
  dump_prog(f, "m", m.m_prog);
  dump_prog(f, "lu", m.lu_prog);
  dump_prog(f, "fwd", m.fwd_prog);
  dump_prog(f, "bwd", m.bwd_prog);
  dump_prog(f, "nudot", m.nudot_prog);
  dump_prog(f, "jt", m.jt_prog);
  dump_prog(f, "fwdT", m.fwdT_prog);
  dump_prog(f, "bwdT", m.bwdT_prog);
  std::fclose(f);
  return 0;
}
