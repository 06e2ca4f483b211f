// Oracle: a plain, slow, single-threaded CPU restatement of the XZZX
// simulated-annealing decoder (arXiv:2509.17837).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark load this library.  It shares no code, header,
// table or constant generator with the CUDA path; both sides are written
// independently from the same definitions.  The product path never calls it.
//
// Representation: one byte per data qubit holding its Pauli as two bits,
// X bit high and Z bit low (I=0, Z=1, X=2, Y=3), the encoding of the footnote
// to Eq. (energy).  Multiplying two Paulis up to phase is XOR of these bytes.
//
// Every function cites the passage of the paper it restates.  Where the paper
// is silent or the problem statement fixes a different form, the reading taken
// is stated beside the code.  No blocking, fusion or reordering beyond what the
// definitions state.
//
// Parity pins live in tests/test_oracle_*.py.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Pauli helpers (Sec. "Principles of error detection and correction").
// ---------------------------------------------------------------------------
const uint8_t PI_ = 0, PZ = 1, PX = 2, PY = 3;

// 1 if the two single-qubit Paulis anticommute (Eq. G_f_comm_anticomm).
int anticommute(uint8_t p, uint8_t q) {
  int px = (p >> 1) & 1, pz = p & 1, qx = (q >> 1) & 1, qz = q & 1;
  return (px & qz) ^ (pz & qx);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).
// The paper only says "pseudorandom numbers"; the generator is fixed here so
// that every draw is a pure function of (seed, counter).
// ---------------------------------------------------------------------------
struct Draw4 {
  uint32_t v[4];
};

Draw4 philox4x32_10(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
  uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  Draw4 out;
  out.v[0] = x0;
  out.v[1] = x1;
  out.v[2] = x2;
  out.v[3] = x3;
  return out;
}

// Purposes of the draws, kept in the top counter word.
const uint32_t TAG_NOISE = 1, TAG_GREEDY = 2, TAG_SA = 3;

// ---------------------------------------------------------------------------
// The rotated XZZX code (Sec. "The XZZX code", Eq. stabilizer_generator).
//
// Reading: the problem statement asks for the rotated d x d layout (d^2 data
// qubits, d^2-1 generators, weight 2 on the boundary).  Qubit (r,c) has index
// r*d+c.  Face (a,b) has corners TL=(a,b), TR=(a,b+1), BL=(a+1,b),
// BR=(a+1,b+1), and G_f = X_TL Z_TR Z_BL X_BR (the paper's
// X_left Z_up Z_down X_right turned by 45 degrees), truncated to the corners
// inside the lattice.  Faces: bulk a,b in [0,d-2]; top a=-1 with b odd;
// bottom a=d-1 with b even; left b=-1 with a even; right b=d-1 with a odd.
// ---------------------------------------------------------------------------
//
// The planar layout (the paper's own lattice, Sec. "The XZZX code"): sites
// (r, c) of a (2d-1) x (2d-1) grid, data qubits where r+c is even
// (d^2 + (d-1)^2 of them), faces where r+c is odd (2d(d-1)).  Face (i, j)
// has corners left=(i,j-1), up=(i-1,j), down=(i+1,j), right=(i,j+1) and
// G_f = X_left Z_up Z_down X_right (Eq. stabilizer_generator), truncated to
// the three corners inside the grid on the boundary.  Qubit (r, c) has index
// (r>>1)(2d-1) + (r odd ? d : 0) + (c>>1), i.e. row-major over the qubit sites.
// ---------------------------------------------------------------------------
const int LAYOUT_ROTATED = 0, LAYOUT_PLANAR = 1;

struct Face {
  int a, b;       // rotated: face (a, b); planar: face site (i, j)
  int colour4;    // sweep colour: four classes of pairwise disjoint generators
  int colour2;    // decoding-graph colour
  int ia, ib;     // coordinates of the face's SA draw inside its colour
  int corner[4];  // qubit of the X, Z, Z, X corner (rotated TL,TR,BL,BR; planar left,up,down,right) or -1
};

const uint8_t CORNER_PAULI[4] = {PX, PZ, PZ, PX};

struct Code {
  int d = 0;
  int layout = LAYOUT_ROTATED;
  int nq = 0;
  std::vector<Face> faces;       // sorted into the stabilizer index order
  std::vector<int> face_at;      // face coordinates -> index or -1
  std::vector<uint8_t> LX, LZ;   // logical operators, one Pauli per qubit
  int colour_start[5];           // faces of colour c are [start[c], start[c+1])

  int face_index(int a, int b) const {
    if (layout == LAYOUT_PLANAR) {
      const int g = 2 * d - 1;
      if (a < 0 || a >= g || b < 0 || b >= g) return -1;
      return face_at[a * g + b];
    }
    if (a < -1 || a > d - 1 || b < -1 || b > d - 1) return -1;
    return face_at[(a + 1) * (d + 1) + (b + 1)];
  }
  // Index of the data qubit at (r, c), or -1 when there is none.
  int qubit(int r, int c) const {
    if (layout == LAYOUT_PLANAR) {
      const int g = 2 * d - 1;
      if (r < 0 || r >= g || c < 0 || c >= g || ((r + c) & 1)) return -1;
      return (r >> 1) * g + ((r & 1) ? d : 0) + (c >> 1);
    }
    return (r >= 0 && r < d && c >= 0 && c < d) ? r * d + c : -1;
  }
  bool qubit_in(int r, int c) const { return qubit(r, c) >= 0; }
};

bool face_present(int d, int a, int b) {
  bool ain = a >= 0 && a <= d - 2, bin = b >= 0 && b <= d - 2;
  if (ain && bin) return true;                         // bulk
  if (a == -1 && bin && (b & 1) == 1) return true;     // top
  if (a == d - 1 && bin && (b & 1) == 0) return true;  // bottom
  if (b == -1 && ain && (a & 1) == 0) return true;     // left
  if (b == d - 1 && ain && (a & 1) == 1) return true;  // right
  return false;
}

bool build_planar(int d, Code& code);

bool build_code(int d, Code& code) {
  if (d < 3 || d % 2 == 0 || d > 255) return false;
  code.d = d;
  code.layout = LAYOUT_ROTATED;
  code.nq = d * d;
  code.faces.clear();
  for (int a = -1; a <= d - 1; ++a) {
    for (int b = -1; b <= d - 1; ++b) {
      if (!face_present(d, a, b)) continue;
      Face f;
      f.a = a;
      f.b = b;
      f.colour4 = (a & 1) | ((b & 1) << 1);
      f.colour2 = (a + b) & 1;
      f.ia = (a + 1) >> 1;
      f.ib = (b + 1) >> 1;
      const int rr[4] = {a, a, a + 1, a + 1};
      const int cc[4] = {b, b + 1, b, b + 1};
      for (int k = 0; k < 4; ++k)
        f.corner[k] = (rr[k] >= 0 && rr[k] < d && cc[k] >= 0 && cc[k] < d) ? rr[k] * d + cc[k] : -1;
      code.faces.push_back(f);
    }
  }
  std::stable_sort(code.faces.begin(), code.faces.end(), [](const Face& x, const Face& y) {
    if (x.colour4 != y.colour4) return x.colour4 < y.colour4;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
  });
  code.face_at.assign((d + 1) * (d + 1), -1);
  for (int i = 0; i < (int)code.faces.size(); ++i)
    code.face_at[(code.faces[i].a + 1) * (d + 1) + (code.faces[i].b + 1)] = i;
  for (int c = 0; c <= 4; ++c) code.colour_start[c] = 0;
  for (const Face& f : code.faces) code.colour_start[f.colour4 + 1]++;
  for (int c = 0; c < 4; ++c) code.colour_start[c + 1] += code.colour_start[c];
  // L_Z joins the left and right boundaries along row 0; L_X joins top and
  // bottom along column 0 (Sec. "The XZZX code").  The alternation makes each
  // commute with every generator.
  code.LX.assign(code.nq, PI_);
  code.LZ.assign(code.nq, PI_);
  for (int c = 0; c < d; ++c) code.LZ[0 * d + c] = (c % 2 == 0) ? PZ : PX;
  for (int r = 0; r < d; ++r) code.LX[r * d + 0] = (r % 2 == 0) ? PX : PZ;
  return true;
}

// The planar layout.  Sweep colour of face (i, j): (i & 1) | (((i+j-1)/2 & 1) << 1);
// two faces share a qubit only when they differ by (+-1, +-1), (+-2, 0) or
// (0, +-2), and each of those changes the colour.  The decoding-graph colour
// is i & 1 (faces on even rows meet the left and right boundaries, faces on odd
// rows the top and bottom ones).  SA draw coordinates ia = i >> 1, ib = j >> 2
// are distinct within a colour.  Stabilizer index order: (colour4, ib, ia), so
// that the four faces sharing one draw block are consecutive.  L_Z = Z on the
// qubits of row 0 (left to right); L_X = X on the qubits of column 0 (top to
// bottom).
bool build_planar(int d, Code& code) {
  if (d < 3 || d % 2 == 0 || d > 127) return false;
  const int g = 2 * d - 1;
  code.d = d;
  code.layout = LAYOUT_PLANAR;
  code.nq = d * d + (d - 1) * (d - 1);
  code.faces.clear();
  for (int i = 0; i < g; ++i) {
    for (int j = 0; j < g; ++j) {
      if (((i + j) & 1) == 0) continue;
      Face f;
      f.a = i;
      f.b = j;
      f.colour4 = (i & 1) | ((((i + j - 1) >> 1) & 1) << 1);
      f.colour2 = i & 1;
      f.ia = i >> 1;
      f.ib = j >> 2;
      f.corner[0] = code.qubit(i, j - 1);
      f.corner[1] = code.qubit(i - 1, j);
      f.corner[2] = code.qubit(i + 1, j);
      f.corner[3] = code.qubit(i, j + 1);
      code.faces.push_back(f);
    }
  }
  std::stable_sort(code.faces.begin(), code.faces.end(), [](const Face& x, const Face& y) {
    if (x.colour4 != y.colour4) return x.colour4 < y.colour4;
    if (x.ib != y.ib) return x.ib < y.ib;
    return x.ia < y.ia;
  });
  code.face_at.assign(g * g, -1);
  for (int k = 0; k < (int)code.faces.size(); ++k) code.face_at[code.faces[k].a * g + code.faces[k].b] = k;
  for (int c = 0; c <= 4; ++c) code.colour_start[c] = 0;
  for (const Face& f : code.faces) code.colour_start[f.colour4 + 1]++;
  for (int c = 0; c < 4; ++c) code.colour_start[c + 1] += code.colour_start[c];
  code.LX.assign(code.nq, PI_);
  code.LZ.assign(code.nq, PI_);
  for (int c = 0; c < g; c += 2) code.LZ[code.qubit(0, c)] = PZ;
  for (int r = 0; r < g; r += 2) code.LX[code.qubit(r, 0)] = PX;
  return true;
}

// Syndrome bit of every face (Eq. G_f_comm_anticomm).
std::vector<uint8_t> syndrome(const Code& code, const std::vector<uint8_t>& C) {
  std::vector<uint8_t> s(code.faces.size(), 0);
  for (size_t f = 0; f < code.faces.size(); ++f) {
    int bit = 0;
    for (int k = 0; k < 4; ++k) {
      int q = code.faces[f].corner[k];
      if (q >= 0) bit ^= anticommute(CORNER_PAULI[k], C[q]);
    }
    s[f] = (uint8_t)bit;
  }
  return s;
}

// C <- C * G_f (footnote on bitwise XOR of the two-bit representation).
void apply_generator(const Code& code, int f, std::vector<uint8_t>& C) {
  for (int k = 0; k < 4; ++k) {
    int q = code.faces[f].corner[k];
    if (q >= 0) C[q] ^= CORNER_PAULI[k];
  }
}

// Logical class of a configuration: bit 0 = anticommutes with L_Z, bit 1 =
// anticommutes with L_X.  For a trivial-syndrome E: I=0, X=1, Z=2, Y=3
// (Sec. "SA decoder that starts with different reference configurations":
// "determined by checking its commutation relations with L_X and L_Z").
int class_bits(const Code& code, const std::vector<uint8_t>& E) {
  int a = 0, b = 0;
  for (int q = 0; q < code.nq; ++q) {
    a ^= anticommute(E[q], code.LZ[q]);
    b ^= anticommute(E[q], code.LX[q]);
  }
  return a | (b << 1);
}

// Pauli index order used for P in {I,X,Y,Z} <-> class bits.
const int INDEX_TO_BITS[4] = {0, 1, 3, 2};
const int BITS_TO_INDEX[4] = {0, 1, 3, 2};

std::vector<uint8_t> logical_config(const Code& code, int P_index) {
  std::vector<uint8_t> L(code.nq, PI_);
  int bits = INDEX_TO_BITS[P_index];
  for (int q = 0; q < code.nq; ++q) {
    if (bits & 1) L[q] ^= code.LX[q];  // an X-class factor
    if (bits & 2) L[q] ^= code.LZ[q];  // a Z-class factor
  }
  return L;
}

// ---------------------------------------------------------------------------
// Noise and energies (Eqs. noise_map, prob_C, coeff_in_energy, energy).
//
// Reading: energies are integers W_P = llround(scale * -ln(p_P/(1-p))),
// i.e. scale * beta_N * alpha_P, so that the Nishimori point is beta = 1.
// Matching weights follow Eq. coeff_in_distance with the same rounding.
// ---------------------------------------------------------------------------
struct Noise {
  double px, py, pz;
  int32_t scale;
  int32_t W[4];    // indexed by the two-bit Pauli: I, Z, X, Y
  int32_t Wt_x, Wt_z;
};

bool make_noise(double px, double py, double pz, int32_t scale, Noise& n) {
  if (!(px > 0.0) || !(py > 0.0) || !(pz > 0.0) || scale <= 0) return false;
  double p = px + py + pz;
  if (!(p < 0.5)) return false;
  n.px = px;
  n.py = py;
  n.pz = pz;
  n.scale = scale;
  double s = (double)scale;
  n.W[PI_] = 0;
  n.W[PX] = (int32_t)std::llround(s * -std::log(px / (1.0 - p)));
  n.W[PY] = (int32_t)std::llround(s * -std::log(py / (1.0 - p)));
  n.W[PZ] = (int32_t)std::llround(s * -std::log(pz / (1.0 - p)));
  n.Wt_x = (int32_t)std::llround(s * -std::log((px + py) / (1.0 - p)));
  n.Wt_z = (int32_t)std::llround(s * -std::log((pz + py) / (1.0 - p)));
  return true;
}

// Eq. energy in integer units.
int64_t energy(const Noise& n, const std::vector<uint8_t>& C) {
  int64_t e = 0;
  for (uint8_t s : C) e += n.W[s];
  return e;
}

// Code-capacity sampling (Sec. "Simulation setting"): each qubit independently
// X, Y or Z with probabilities px, py, pz.  The uniform draw u of qubit q is
// compared with floor(p*2^32) thresholds.
std::vector<uint8_t> sample_error(const Code& code, const Noise& n, uint64_t seed, uint64_t shot) {
  uint64_t Tx = (uint64_t)std::floor(std::ldexp(n.px, 32));
  uint64_t Ty = (uint64_t)std::floor(std::ldexp(n.py, 32));
  uint64_t Tz = (uint64_t)std::floor(std::ldexp(n.pz, 32));
  std::vector<uint8_t> C(code.nq, PI_);
  for (int q = 0; q < code.nq; ++q) {
    Draw4 r = philox4x32_10(seed, (uint32_t)(q >> 2), (uint32_t)shot, (uint32_t)(shot >> 32), TAG_NOISE);
    uint64_t u = r.v[q & 3];
    if (u < Tx)
      C[q] = PX;
    else if (u < Tx + Ty)
      C[q] = PY;
    else if (u < Tx + Ty + Tz)
      C[q] = PZ;
    else
      C[q] = PI_;
  }
  return C;
}

// ---------------------------------------------------------------------------
// Decoding graphs (Sec. "Principles of error detection and correction").
// Rotated: the Z component of qubit (r,c) is an edge between faces (r-1,c-1)
// and (r,c); its X component an edge between faces (r-1,c) and (r,c-1).
// Planar: the Z component of qubit (r,c) is the horizontal edge between faces
// (r,c-1) and (r,c+1), its X component the vertical edge between (r-1,c) and
// (r+1,c).  A missing end face makes the edge a boundary edge.  Z edges weigh
// Wt_z, X edges Wt_x (Eqs. distance_u_v_internal, coeff_in_distance).
// ---------------------------------------------------------------------------
const int BOUNDARY = 0xFFFF;

// End faces (or -1) of the Z edge (e = 0) and the X edge (e = 1) of the qubit
// at site (r, c).
void qubit_edge_ends(const Code& code, int r, int c, int ends[2][2]) {
  if (code.layout == LAYOUT_PLANAR) {
    ends[0][0] = code.face_index(r, c - 1);
    ends[0][1] = code.face_index(r, c + 1);
    ends[1][0] = code.face_index(r - 1, c);
    ends[1][1] = code.face_index(r + 1, c);
    return;
  }
  ends[0][0] = code.face_index(r - 1, c - 1);
  ends[0][1] = code.face_index(r, c);
  ends[1][0] = code.face_index(r - 1, c);
  ends[1][1] = code.face_index(r, c - 1);
}

// The four edges of a face in walking order: Z, Z, X, X.  Gives the face at
// the other end (its coordinates) and the crossed qubit's site.  Rotated:
// Z(+1,+1), Z(-1,-1), X(+1,-1), X(-1,+1), crossing qubit (max a, max b).
// Planar: Z right, Z left (crossing (i, j+-1)), X down, X up (crossing (i+-1, j)).
void face_step(const Code& code, int a, int b, int e, int& na, int& nb, int& qr, int& qc) {
  if (code.layout == LAYOUT_PLANAR) {
    const int di[4] = {0, 0, 1, -1}, dj[4] = {1, -1, 0, 0};
    na = a + 2 * di[e];
    nb = b + 2 * dj[e];
    qr = a + di[e];
    qc = b + dj[e];
    return;
  }
  const int da[4] = {1, -1, 1, -1};
  const int db[4] = {1, -1, -1, 1};
  na = a + da[e];
  nb = b + db[e];
  qr = std::max(a, na);
  qc = std::max(b, nb);
}

// Shortest distance from every face to the open boundary of its decoding
// graph (the w(u,b) of Eq. distance_u_boundary).  Reading: the paper's closed
// forms are for its own lattice; for the rotated layout the distance is taken
// as the graph shortest path, computed here by plain Dijkstra.
std::vector<int64_t> boundary_distance(const Code& code, const Noise& n) {
  const int nf = (int)code.faces.size();
  const int64_t INF = (int64_t)1 << 60;
  // adjacency: (neighbour face or -1 for the boundary, weight)
  std::vector<std::vector<std::pair<int, int64_t>>> adj(nf);
  std::vector<int64_t> to_boundary(nf, INF);
  const int g = code.layout == LAYOUT_PLANAR ? 2 * code.d - 1 : code.d;
  for (int r = 0; r < g; ++r) {
    for (int c = 0; c < g; ++c) {
      if (!code.qubit_in(r, c)) continue;
      int ends[2][2];
      qubit_edge_ends(code, r, c, ends);
      int64_t w[2] = {n.Wt_z, n.Wt_x};
      for (int e = 0; e < 2; ++e) {
        int f1 = ends[e][0], f2 = ends[e][1];
        if (f1 >= 0 && f2 >= 0) {
          adj[f1].push_back({f2, w[e]});
          adj[f2].push_back({f1, w[e]});
        } else if (f1 >= 0) {
          to_boundary[f1] = std::min(to_boundary[f1], w[e]);
        } else if (f2 >= 0) {
          to_boundary[f2] = std::min(to_boundary[f2], w[e]);
        }
      }
    }
  }
  std::vector<int64_t> dist = to_boundary;
  std::vector<char> done(nf, 0);
  for (int it = 0; it < nf; ++it) {
    int best = -1;
    for (int f = 0; f < nf; ++f)
      if (!done[f] && (best < 0 || dist[f] < dist[best])) best = f;
    if (best < 0 || dist[best] >= INF) break;
    done[best] = 1;
    for (auto& e : adj[best])
      if (dist[best] + e.second < dist[e.first]) dist[e.first] = dist[best] + e.second;
  }
  return dist;
}

// Weighted Manhattan distance of Eq. distance_u_v_internal.  Rotated
// coordinates: a Z step changes a+b by 2, an X step changes a-b by 2.  Planar:
// a Z step changes j by 2, an X step changes i by 2.
int64_t internal_distance(const Code& code, const Noise& n, int u, int v) {
  const Face& fu = code.faces[u];
  const Face& fv = code.faces[v];
  if (code.layout == LAYOUT_PLANAR)
    return n.Wt_z * (std::llabs((int64_t)fu.b - fv.b) / 2) + n.Wt_x * (std::llabs((int64_t)fu.a - fv.a) / 2);
  int64_t ds = std::llabs((int64_t)(fu.a + fu.b) - (fv.a + fv.b)) / 2;
  int64_t dd = std::llabs((int64_t)(fu.a - fu.b) - (fv.a - fv.b)) / 2;
  return n.Wt_z * ds + n.Wt_x * dd;
}

// Toggle one component of a qubit: a Z step flips its Z bit, an X step its X bit.
void toggle(std::vector<uint8_t>& R, int q, bool z_step) { R[q] ^= z_step ? PZ : PX; }

// "Add to C the edges along a path connecting u and v with the weight w(u,v)"
// (Alg. 5).  Reading: edges are added modulo two, and the minimal path is the
// canonical walk that takes a Z step toward v whenever one is still needed and
// both the next face and the crossed qubit exist, else an X step.
bool walk_internal_planar(const Code& code, int u, int v, std::vector<uint8_t>& R);

bool walk_internal(const Code& code, int u, int v, std::vector<uint8_t>& R) {
  if (code.layout == LAYOUT_PLANAR) return walk_internal_planar(code, u, v, R);
  int a = code.faces[u].a, b = code.faces[u].b;
  const int ta = code.faces[v].a, tb = code.faces[v].b;
  int guard = 4 * code.d * code.d + 8;
  while (a != ta || b != tb) {
    if (--guard < 0) return false;
    int ds = (ta + tb) - (a + b);
    int dd = (ta - tb) - (a - b);
    bool moved = false;
    if (ds != 0) {
      int s = ds > 0 ? 1 : -1;
      int na = a + s, nb = b + s;
      int qr = std::max(a, na), qc = std::max(b, nb);
      if (code.face_index(na, nb) >= 0 && code.qubit_in(qr, qc)) {
        toggle(R, qr * code.d + qc, true);
        a = na;
        b = nb;
        moved = true;
      }
    }
    if (!moved && dd != 0) {
      int s = dd > 0 ? 1 : -1;
      int na = a + s, nb = b - s;
      int qr = std::max(a, na), qc = std::max(b, nb);
      if (code.face_index(na, nb) >= 0 && code.qubit_in(qr, qc)) {
        toggle(R, qr * code.d + qc, false);
        a = na;
        b = nb;
        moved = true;
      }
    }
    if (!moved) return false;
  }
  return true;
}

// Planar form of the same canonical walk: a horizontal Z step toward v while
// the columns differ, then vertical X steps (every face between two faces of
// one decoding-graph colour exists on the planar grid).
bool walk_internal_planar(const Code& code, int u, int v, std::vector<uint8_t>& R) {
  int i = code.faces[u].a, j = code.faces[u].b;
  const int ti = code.faces[v].a, tj = code.faces[v].b;
  if (((ti - i) & 1) || ((tj - j) & 1)) return false;
  while (j != tj) {
    const int s = tj > j ? 1 : -1;
    if (code.face_index(i, j + 2 * s) < 0 || !code.qubit_in(i, j + s)) return false;
    toggle(R, code.qubit(i, j + s), true);
    j += 2 * s;
  }
  while (i != ti) {
    const int s = ti > i ? 1 : -1;
    if (code.face_index(i + 2 * s, j) < 0 || !code.qubit_in(i + s, j)) return false;
    toggle(R, code.qubit(i + s, j), false);
    i += 2 * s;
  }
  return true;
}

// Walk a face to its open boundary along a shortest path: at each face take
// the first incident edge, in the walking order of face_step, that lowers the
// remaining boundary distance by exactly its own weight.
bool walk_to_boundary(const Code& code, const Noise& n, const std::vector<int64_t>& wb, int u,
                      std::vector<uint8_t>& R) {
  int cur = u;
  int guard = 8 * code.d * code.d + 8;
  while (true) {
    if (--guard < 0) return false;
    int a = code.faces[cur].a, b = code.faces[cur].b;
    bool moved = false;
    for (int e = 0; e < 4 && !moved; ++e) {
      bool z_step = e < 2;
      int na, nb, qr, qc;
      face_step(code, a, b, e, na, nb, qr, qc);
      if (!code.qubit_in(qr, qc)) continue;
      int64_t w = z_step ? n.Wt_z : n.Wt_x;
      int nf = code.face_index(na, nb);
      if (nf < 0) {
        if (w == wb[cur]) {
          toggle(R, code.qubit(qr, qc), z_step);
          return true;
        }
      } else if (wb[nf] + w == wb[cur]) {
        toggle(R, code.qubit(qr, qc), z_step);
        cur = nf;
        moved = true;
      }
    }
    if (!moved) return false;
  }
}

struct Pair {
  int64_t w;
  uint32_t key;
  int u, v;
};

// Greedy matching of one decoding-graph colour: Alg. 5 (randomised = 0) and
// Alg. 6 (randomised = 1).  Reading of Alg. 6: picking uniformly among the
// remaining minimum-weight pairs until none is left, then recomputing the
// minimum, is the same distribution as scanning all pairs in the order
// (w, key, u, v) with a fresh uniform key per pair and keeping a pair when both
// ends are still free.  Alg. 5 leaves ties unspecified; key = 0 makes them
// lexicographic in (u, v).  u < v are stabilizer indices; the virtual boundary
// vertex b (appended when the defect count is odd) is v = 0xFFFF.
bool greedy_colour(const Code& code, const Noise& n, const std::vector<int64_t>& wb,
                   const std::vector<uint8_t>& S, int colour2, uint64_t seed, uint64_t shot,
                   int restart, int randomised, std::vector<uint8_t>& R, int64_t& weight_sum) {
  std::vector<int> D;
  for (int f = 0; f < (int)code.faces.size(); ++f)
    if (code.faces[f].colour2 == colour2 && S[f]) D.push_back(f);
  auto key_of = [&](int u, int v) -> uint32_t {
    if (!randomised) return 0u;
    Draw4 r = philox4x32_10(seed, (uint32_t)u | ((uint32_t)v << 16), (uint32_t)restart, (uint32_t)shot,
                            TAG_GREEDY | ((uint32_t)(shot >> 32) << 8));
    return r.v[0];
  };
  std::vector<Pair> K;
  for (size_t i = 0; i < D.size(); ++i) {
    for (size_t j = i + 1; j < D.size(); ++j) {
      int u = D[i], v = D[j];
      int64_t w = std::min(internal_distance(code, n, u, v), wb[u] + wb[v]);  // Eq. distance_u_v_def_new
      K.push_back({w, key_of(u, v), u, v});
    }
  }
  if (D.size() % 2 == 1)
    for (int u : D) K.push_back({wb[u], key_of(u, BOUNDARY), u, BOUNDARY});
  std::sort(K.begin(), K.end(), [](const Pair& x, const Pair& y) {
    if (x.w != y.w) return x.w < y.w;
    if (x.key != y.key) return x.key < y.key;
    if (x.u != y.u) return x.u < y.u;
    return x.v < y.v;
  });
  std::vector<char> matched(code.faces.size(), 0);
  bool boundary_matched = false;
  for (const Pair& p : K) {
    bool v_free = (p.v == BOUNDARY) ? !boundary_matched : !matched[p.v];
    if (matched[p.u] || !v_free) continue;
    matched[p.u] = 1;
    if (p.v == BOUNDARY)
      boundary_matched = true;
    else
      matched[p.v] = 1;
    weight_sum += p.w;
    bool ok;
    if (p.v == BOUNDARY) {
      ok = walk_to_boundary(code, n, wb, p.u, R);
    } else if (internal_distance(code, n, p.u, p.v) <= wb[p.u] + wb[p.v]) {
      ok = walk_internal(code, p.u, p.v, R);  // ties between the two forms take the internal path
    } else {
      ok = walk_to_boundary(code, n, wb, p.u, R) && walk_to_boundary(code, n, wb, p.v, R);
    }
    if (!ok) return false;
  }
  return true;
}

// Initial reference configurations (Sec. "Effect of initial error
// configuration on SA performance"): mode 0 = greedy matching with
// lexicographic ties (Alg. 5; every restart gets the same R, as in Alg. 1),
// mode 1 = greedy matching with random tie-breaking (Alg. 6), mode 2 =
// "boundary": every defect joined to the nearer boundary of its decoding
// graph (a shortest path to the open boundary).
const int INIT_GREEDY = 0, INIT_GREEDY_RANDOM = 1, INIT_BOUNDARY = 2;

bool greedy(const Code& code, const Noise& n, const std::vector<uint8_t>& S, uint64_t seed, uint64_t shot,
            int restart, int mode, std::vector<uint8_t>& R, int64_t& weight_sum) {
  std::vector<int64_t> wb = boundary_distance(code, n);
  R.assign(code.nq, PI_);
  weight_sum = 0;
  if (mode == INIT_BOUNDARY) {
    for (int f = 0; f < (int)code.faces.size(); ++f) {
      if (!S[f]) continue;
      weight_sum += wb[f];
      if (!walk_to_boundary(code, n, wb, f, R)) return false;
    }
    return true;
  }
  for (int colour2 = 0; colour2 < 2; ++colour2)
    if (!greedy_colour(code, n, wb, S, colour2, seed, shot, restart, mode == INIT_GREEDY_RANDOM ? 1 : 0, R,
                       weight_sum))
      return false;
  return true;
}

// ---------------------------------------------------------------------------
// Schedules and acceptance (Eqs. beta_i, beta_ratio; Alg. 3).
//
// Reading: the problem statement fixes a linear schedule beta_t = beta0 +
// (beta1-beta0) t/(N-1), t = 0..N-1 (beta0 when N = 1); the paper's
// logarithmic schedule (Eq. beta_i with beta_init = beta0, beta_final = beta1)
// is the second kind.  In the integer energy units beta is measured in units
// of beta_N.  Acceptance r < min(1, exp(-beta dE)) with r = u/2^32 is taken in
// integers: accept when dE <= 0 or u < T, T = min(2^32-1, floor(2^32 exp(-beta
// dE/scale))) evaluated in FP64.
// ---------------------------------------------------------------------------
const int SCHED_LINEAR = 0, SCHED_PAPER_LOG = 1;

double beta_at(int kind, int n_sweeps, double beta0, double beta1, int t) {
  if (kind == SCHED_LINEAR) {
    if (n_sweeps <= 1) return beta0;
    return beta0 + (beta1 - beta0) * (double)t / (double)(n_sweeps - 1);
  }
  double gamma = n_sweeps >= 2 ? (beta1 / beta0 - 1.0) / std::log((double)n_sweeps) : 0.0;
  return beta0 * (1.0 + gamma * std::log((double)(t + 1)));
}

uint32_t accept_threshold(double beta, int32_t dE, int32_t scale) {
  double x = beta * (double)dE / (double)scale;
  double v = std::ldexp(std::exp(-x), 32);
  if (v >= 4294967295.0) return 0xFFFFFFFFu;
  return (uint32_t)v;
}

struct Schedule {
  int kind;
  int n_sweeps;
  double beta0, beta1;
};

// Alg. 2 with the Metropolis step of Alg. 3 (R5, R6 readings):
//  * a sweep visits the generators colour by colour (colours 0..3, index
//    order within a colour), each once, instead of N_stab uniformly random
//    picks; each single-generator Metropolis update keeps the Boltzmann
//    distribution stationary either way;
//  * the minimum energy and its configuration are recorded at the start and
//    after every colour phase (strict improvement keeps the earliest).
// The draw for the face (a, b) of colour c at sweep t of chain `chain` is lane
// (ia & 3) of Philox(seed; (c<<16)|(ib<<8)|(ia>>2), t, chain_lo,
// TAG_SA|chain_hi<<8) with ia = (a+1)>>1 and ib = (b+1)>>1 (distinct within a
// colour, since a colour fixes the parities of a and b).
struct ChainResult {
  int32_t best_E;
  int32_t final_E;
  std::vector<uint8_t> best, final_cfg;
};

// Variants of Alg. 2 kept for comparison with the readings above:
//   order 1: each sweep makes N_stab attempts on generators picked uniformly
//            at random, as Alg. 3 states (site draw and acceptance draw from
//            Philox(seed; k>>1, t, chain_lo, TAG_SITE|chain_hi<<8), lanes
//            2(k&1) and 2(k&1)+1 for attempt k);
//   emin 1:  the minimum is updated after every attempt, as Alg. 2 states.
const int ORDER_COLOUR = 0, ORDER_RANDOM_SITE = 1;
const int EMIN_PER_PHASE = 0, EMIN_PER_ATTEMPT = 1;
const uint32_t TAG_SITE = 4;

ChainResult anneal_chain_variant(const Code& code, const Noise& n, const Schedule& sch, uint64_t seed, uint64_t chain,
                                 const std::vector<uint8_t>& init, int order, int emin, int32_t* trace_E);

ChainResult anneal_chain(const Code& code, const Noise& n, const Schedule& sch, uint64_t seed, uint64_t chain,
                         const std::vector<uint8_t>& init, int32_t* trace_E) {
  return anneal_chain_variant(code, n, sch, seed, chain, init, ORDER_COLOUR, EMIN_PER_PHASE, trace_E);
}

ChainResult anneal_chain_variant(const Code& code, const Noise& n, const Schedule& sch, uint64_t seed, uint64_t chain,
                                 const std::vector<uint8_t>& init, int order, int emin, int32_t* trace_E) {
  std::vector<uint8_t> C = init;
  int64_t E = energy(n, C);
  int64_t E_best = E;
  std::vector<uint8_t> best = C;
  const uint32_t chain_lo = (uint32_t)chain, chain_hi = (uint32_t)(chain >> 32);
  const int m = (int)code.faces.size();
  for (int t = 0; t < sch.n_sweeps; ++t) {
    double beta = beta_at(sch.kind, sch.n_sweeps, sch.beta0, sch.beta1, t);
    if (order == ORDER_RANDOM_SITE) {
      for (int k = 0; k < m; ++k) {
        Draw4 r = philox4x32_10(seed, (uint32_t)(k >> 1), (uint32_t)t, chain_lo, TAG_SITE | (chain_hi << 8));
        const int f = (int)(((uint64_t)r.v[2 * (k & 1)] * (uint64_t)m) >> 32);
        int64_t dE = 0;
        for (int c = 0; c < 4; ++c) {
          int q = code.faces[f].corner[c];
          if (q < 0) continue;
          dE += (int64_t)n.W[C[q] ^ CORNER_PAULI[c]] - (int64_t)n.W[C[q]];
        }
        const bool accept = dE <= 0 || r.v[2 * (k & 1) + 1] < accept_threshold(beta, (int32_t)dE, n.scale);
        if (accept) {
          apply_generator(code, f, C);
          E += dE;
        }
        if (emin == EMIN_PER_ATTEMPT && E < E_best) {
          E_best = E;
          best = C;
        }
      }
      if (emin == EMIN_PER_PHASE && E < E_best) {
        E_best = E;
        best = C;
      }
      if (trace_E) trace_E[t] = (int32_t)E;
      continue;
    }
    for (int colour = 0; colour < 4; ++colour) {
      for (int f = code.colour_start[colour]; f < code.colour_start[colour + 1]; ++f) {
        const int ia = code.faces[f].ia, ib = code.faces[f].ib;
        // dE = H(C G_f) - H(C), summed over the support of G_f.
        int64_t dE = 0;
        for (int k = 0; k < 4; ++k) {
          int q = code.faces[f].corner[k];
          if (q < 0) continue;
          dE += (int64_t)n.W[C[q] ^ CORNER_PAULI[k]] - (int64_t)n.W[C[q]];
        }
        bool accept;
        if (dE <= 0) {
          accept = true;
        } else {
          Draw4 r = philox4x32_10(seed, ((uint32_t)colour << 16) | ((uint32_t)ib << 8) | (uint32_t)(ia >> 2),
                                  (uint32_t)t, chain_lo, TAG_SA | (chain_hi << 8));
          accept = r.v[ia & 3] < accept_threshold(beta, (int32_t)dE, n.scale);
        }
        if (accept) {
          apply_generator(code, f, C);
          E += dE;
        }
        if (emin == EMIN_PER_ATTEMPT && E < E_best) {
          E_best = E;
          best = C;
        }
      }
      if (E < E_best) {
        E_best = E;
        best = C;
      }
    }
    if (trace_E) trace_E[t] = (int32_t)E;
  }
  ChainResult res;
  res.best_E = (int32_t)E_best;
  res.final_E = (int32_t)E;
  res.best = best;
  res.final_cfg = C;
  return res;
}

// Alg. 7: SA decoder with a fresh randomised greedy reference per restart.
// Chain (i, P) starts from R_i L_P and belongs to coset Q_i P of R_1, where
// [L_Q] = [R_i R_1] (Eq. coset_correspondence).  E_P is the minimum over the
// chains of coset P, P* = argmin with ties broken in the order I, X, Y, Z, and
// the recovery is R_1 L_{P*}.  The chain id of (shot, i, P) is
// (shot * restarts + i) * 4 + P.
struct ShotResult {
  int cls;
  int32_t E4[4];
  std::vector<uint8_t> recovery;
  std::vector<uint8_t> best_cfg;
  std::vector<int32_t> chain_E;
  std::vector<uint8_t> q_bits;
};

bool decode_shot(const Code& code, const Noise& n, const Schedule& sch, uint64_t seed, uint64_t shot, int restarts,
                 int randomised, const std::vector<uint8_t>& S, ShotResult& out) {
  std::vector<std::vector<uint8_t>> R(restarts);
  std::vector<int> cbits(restarts);
  for (int i = 0; i < restarts; ++i) {
    int64_t wsum = 0;
    if (!greedy(code, n, S, seed, shot, i, randomised, R[i], wsum)) return false;
    cbits[i] = class_bits(code, R[i]);
  }
  const int64_t BIG = (int64_t)1 << 40;
  int64_t E_coset[4] = {BIG, BIG, BIG, BIG};
  int best_chain_of[4] = {-1, -1, -1, -1};
  std::vector<std::vector<uint8_t>> cfg(4 * restarts);
  out.chain_E.assign(4 * restarts, 0);
  out.q_bits.assign(restarts, 0);
  for (int i = 0; i < restarts; ++i) {
    int Q = cbits[i] ^ cbits[0];
    out.q_bits[i] = (uint8_t)Q;
    for (int P = 0; P < 4; ++P) {
      std::vector<uint8_t> init = R[i];
      std::vector<uint8_t> L = logical_config(code, P);
      for (int q = 0; q < code.nq; ++q) init[q] ^= L[q];
      uint64_t chain = ((uint64_t)shot * (uint64_t)restarts + (uint64_t)i) * 4u + (uint64_t)P;
      ChainResult cr = anneal_chain(code, n, sch, seed, chain, init, nullptr);
      out.chain_E[i * 4 + P] = cr.best_E;
      cfg[i * 4 + P] = cr.best;
      int coset = BITS_TO_INDEX[Q ^ INDEX_TO_BITS[P]];
      if (cr.best_E < E_coset[coset]) {  // strict: the lowest (i, P) wins ties
        E_coset[coset] = cr.best_E;
        best_chain_of[coset] = i * 4 + P;
      }
    }
  }
  int Pstar = 0;
  for (int P = 1; P < 4; ++P)
    if (E_coset[P] < E_coset[Pstar]) Pstar = P;
  out.cls = Pstar;
  for (int P = 0; P < 4; ++P) out.E4[P] = (int32_t)E_coset[P];
  out.recovery = R[0];
  std::vector<uint8_t> L = logical_config(code, Pstar);
  for (int q = 0; q < code.nq; ++q) out.recovery[q] ^= L[q];
  out.best_cfg = cfg[best_chain_of[Pstar]];
  return true;
}

// Code id: the distance d for the rotated layout, d + 1000 for the planar one.
bool get_code(int id, Code& code) {
  if (id >= 1000) return build_planar(id - 1000, code);
  return build_code(id, code);
}

}  // namespace

// ===========================================================================
// C ABI for the tests (ctypes).  Status: 0 = ok, -1 = bad argument, -2 = an
// internal walk failed (never expected).
// ===========================================================================
extern "C" {

int orc_philox(uint64_t key, const uint32_t* ctr, uint32_t* out) {
  Draw4 r = philox4x32_10(key, ctr[0], ctr[1], ctr[2], ctr[3]);
  for (int i = 0; i < 4; ++i) out[i] = r.v[i];
  return 0;
}

int orc_code_sizes(int d, int* nq, int* nstab, int* colour_start5) {
  Code code;
  if (!get_code(d, code)) return -1;
  *nq = code.nq;
  *nstab = (int)code.faces.size();
  for (int c = 0; c < 5; ++c) colour_start5[c] = code.colour_start[c];
  return 0;
}

// Per stabilizer: a, b, colour4, colour2 and the four corner qubits (or -1).
int orc_code_faces(int d, int32_t* a, int32_t* b, int32_t* colour4, int32_t* colour2, int32_t* corners) {
  Code code;
  if (!get_code(d, code)) return -1;
  for (size_t f = 0; f < code.faces.size(); ++f) {
    a[f] = code.faces[f].a;
    b[f] = code.faces[f].b;
    colour4[f] = code.faces[f].colour4;
    colour2[f] = code.faces[f].colour2;
    for (int k = 0; k < 4; ++k) corners[4 * f + k] = code.faces[f].corner[k];
  }
  return 0;
}

int orc_logicals(int d, uint8_t* LX, uint8_t* LZ) {
  Code code;
  if (!get_code(d, code)) return -1;
  std::memcpy(LX, code.LX.data(), code.nq);
  std::memcpy(LZ, code.LZ.data(), code.nq);
  return 0;
}

// W4 = (W_I, W_Z, W_X, W_Y) by two-bit Pauli; Wt2 = (Wt_x, Wt_z).
int orc_make_noise(double px, double py, double pz, int32_t scale, int32_t* W4, int32_t* Wt2) {
  Noise n;
  if (!make_noise(px, py, pz, scale, n)) return -1;
  for (int i = 0; i < 4; ++i) W4[i] = n.W[i];
  Wt2[0] = n.Wt_x;
  Wt2[1] = n.Wt_z;
  return 0;
}

// Bias conventions: 0 = problem statement (py = p eta/(eta+1), px = pz =
// p/(2(eta+1))), 1 = the paper's px:py:pz = 1:eta:1 (Sec. "Simulation setting").
int orc_noise_from_eta(double p, double eta, int convention, double* pxyz) {
  if (!(p > 0.0) || !(eta > 0.0)) return -1;
  if (convention == 0) {
    pxyz[1] = p * eta / (eta + 1.0);
    pxyz[0] = p / (2.0 * (eta + 1.0));
    pxyz[2] = pxyz[0];
  } else if (convention == 1) {
    pxyz[1] = p * eta / (eta + 2.0);
    pxyz[0] = p / (eta + 2.0);
    pxyz[2] = pxyz[0];
  } else {
    return -1;
  }
  return 0;
}

int orc_sample(int d, double px, double py, double pz, uint64_t seed, uint64_t shot0, int n_shots, uint8_t* err,
               uint8_t* syn) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, 1024, n) || n_shots < 0) return -1;
  const int nq = code.nq, ns = (int)code.faces.size();
  for (int s = 0; s < n_shots; ++s) {
    std::vector<uint8_t> C = sample_error(code, n, seed, shot0 + (uint64_t)s);
    std::vector<uint8_t> S = syndrome(code, C);
    if (err) std::memcpy(err + (size_t)s * nq, C.data(), nq);
    if (syn) std::memcpy(syn + (size_t)s * ns, S.data(), ns);
  }
  return 0;
}

int orc_syndrome(int d, const uint8_t* cfg, uint8_t* syn) {
  Code code;
  if (!get_code(d, code)) return -1;
  std::vector<uint8_t> C(cfg, cfg + code.nq);
  std::vector<uint8_t> S = syndrome(code, C);
  std::memcpy(syn, S.data(), S.size());
  return 0;
}

int orc_class_bits(int d, const uint8_t* cfg) {
  Code code;
  if (!get_code(d, code)) return -1;
  std::vector<uint8_t> C(cfg, cfg + code.nq);
  return class_bits(code, C);
}

int orc_boundary_distance(int d, double px, double py, double pz, int32_t scale, int64_t* wb) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, scale, n)) return -1;
  std::vector<int64_t> v = boundary_distance(code, n);
  std::memcpy(wb, v.data(), v.size() * sizeof(int64_t));
  return 0;
}

int orc_greedy(int d, double px, double py, double pz, int32_t scale, uint64_t seed, uint64_t shot, int restart,
               int randomised, const uint8_t* syn, uint8_t* R_out, int64_t* weight_sum) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, scale, n)) return -1;
  std::vector<uint8_t> S(syn, syn + code.faces.size());
  std::vector<uint8_t> R;
  int64_t w = 0;
  if (!greedy(code, n, S, seed, shot, restart, randomised, R, w)) return -2;
  std::memcpy(R_out, R.data(), code.nq);
  if (weight_sum) *weight_sum = w;
  return 0;
}

int orc_walk_internal(int d, int u, int v, uint8_t* R_out) {
  Code code;
  if (!get_code(d, code)) return -1;
  std::vector<uint8_t> R(code.nq, PI_);
  if (!walk_internal(code, u, v, R)) return -2;
  std::memcpy(R_out, R.data(), code.nq);
  return 0;
}

int orc_walk_boundary(int d, double px, double py, double pz, int32_t scale, int u, uint8_t* R_out) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, scale, n)) return -1;
  std::vector<int64_t> wb = boundary_distance(code, n);
  std::vector<uint8_t> R(code.nq, PI_);
  if (!walk_to_boundary(code, n, wb, u, R)) return -2;
  std::memcpy(R_out, R.data(), code.nq);
  return 0;
}

double orc_beta_at(int kind, int n_sweeps, double beta0, double beta1, int t) {
  return beta_at(kind, n_sweeps, beta0, beta1, t);
}

uint32_t orc_accept_threshold(double beta, int32_t dE, int32_t scale) { return accept_threshold(beta, dE, scale); }

int orc_anneal_chain(int d, double px, double py, double pz, int32_t scale, int kind, int n_sweeps, double beta0,
                     double beta1, uint64_t seed, uint64_t chain, const uint8_t* init, uint8_t* best,
                     int32_t* best_E, uint8_t* final_cfg, int32_t* final_E, int32_t* trace_E) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, scale, n) || n_sweeps < 0) return -1;
  Schedule sch{kind, n_sweeps, beta0, beta1};
  std::vector<uint8_t> C(init, init + code.nq);
  ChainResult r = anneal_chain(code, n, sch, seed, chain, C, trace_E);
  if (best) std::memcpy(best, r.best.data(), code.nq);
  if (best_E) *best_E = r.best_E;
  if (final_cfg) std::memcpy(final_cfg, r.final_cfg.data(), code.nq);
  if (final_E) *final_E = r.final_E;
  return 0;
}

int orc_anneal_chain_variant(int d, double px, double py, double pz, int32_t scale, int kind, int n_sweeps,
                             double beta0, double beta1, uint64_t seed, uint64_t chain, const uint8_t* init,
                             int order, int emin, uint8_t* best, int32_t* best_E, uint8_t* final_cfg,
                             int32_t* final_E, int32_t* trace_E) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, scale, n) || n_sweeps < 0) return -1;
  Schedule sch{kind, n_sweeps, beta0, beta1};
  std::vector<uint8_t> C(init, init + code.nq);
  ChainResult r = anneal_chain_variant(code, n, sch, seed, chain, C, order, emin, trace_E);
  if (best) std::memcpy(best, r.best.data(), code.nq);
  if (best_E) *best_E = r.best_E;
  if (final_cfg) std::memcpy(final_cfg, r.final_cfg.data(), code.nq);
  if (final_E) *final_E = r.final_E;
  return 0;
}

// Decode n_shots syndromes (row s of syn belongs to shot shot0+s).  Optional
// outputs may be null.  err, when given, yields the failure flag
// [C_true C] != [I] (Sec. "Simulation setting").
int orc_decode(int d, double px, double py, double pz, int32_t scale, int kind, int n_sweeps, double beta0,
               double beta1, uint64_t seed, uint64_t shot0, int n_shots, int restarts, int randomised,
               const uint8_t* syn, const uint8_t* err, uint8_t* cls, int32_t* E4, uint8_t* recovery,
               uint8_t* best_cfg, uint8_t* fail, int32_t* chain_E, uint8_t* q_bits) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, scale, n) || n_shots < 0 || restarts < 1) return -1;
  Schedule sch{kind, n_sweeps, beta0, beta1};
  const int nq = code.nq, ns = (int)code.faces.size();
  for (int s = 0; s < n_shots; ++s) {
    std::vector<uint8_t> S(syn + (size_t)s * ns, syn + (size_t)(s + 1) * ns);
    ShotResult r;
    if (!decode_shot(code, n, sch, seed, shot0 + (uint64_t)s, restarts, randomised, S, r)) return -2;
    if (cls) cls[s] = (uint8_t)r.cls;
    if (E4)
      for (int P = 0; P < 4; ++P) E4[4 * s + P] = r.E4[P];
    if (recovery) std::memcpy(recovery + (size_t)s * nq, r.recovery.data(), nq);
    if (best_cfg) std::memcpy(best_cfg + (size_t)s * nq, r.best_cfg.data(), nq);
    if (chain_E) std::memcpy(chain_E + (size_t)s * 4 * restarts, r.chain_E.data(), 4 * restarts * sizeof(int32_t));
    if (q_bits) std::memcpy(q_bits + (size_t)s * restarts, r.q_bits.data(), restarts);
    if (fail && err) {
      std::vector<uint8_t> prod(err + (size_t)s * nq, err + (size_t)(s + 1) * nq);
      for (int q = 0; q < nq; ++q) prod[q] ^= r.recovery[q];
      fail[s] = class_bits(code, prod) != 0;
    }
  }
  return 0;
}

// Exact coset minima E^min_P (Eq. min_energy) by enumerating the whole
// stabilizer group in Gray-code order, for P in I, X, Y, Z relative to R.
int orc_bruteforce(int d, double px, double py, double pz, int32_t scale, const uint8_t* R, int32_t* Emin4) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, scale, n)) return -1;
  const int m = (int)code.faces.size();
  if (m > 30) return -1;
  for (int P = 0; P < 4; ++P) {
    std::vector<uint8_t> C(R, R + code.nq);
    std::vector<uint8_t> L = logical_config(code, P);
    for (int q = 0; q < code.nq; ++q) C[q] ^= L[q];
    int64_t E = energy(n, C);
    int64_t best = E;
    const uint64_t total = (uint64_t)1 << m;
    for (uint64_t k = 1; k < total; ++k) {
      int g = __builtin_ctzll(k);
      for (int c = 0; c < 4; ++c) {
        int q = code.faces[g].corner[c];
        if (q < 0) continue;
        E += (int64_t)n.W[C[q] ^ CORNER_PAULI[c]] - (int64_t)n.W[C[q]];
        C[q] ^= CORNER_PAULI[c];
      }
      if (E < best) best = E;
    }
    Emin4[P] = (int32_t)best;
  }
  return 0;
}

// Energies of all 2^m configurations of one coset (for the detailed-balance pin).
int orc_coset_energies(int d, double px, double py, double pz, int32_t scale, const uint8_t* start, int32_t* E_out) {
  Code code;
  Noise n;
  if (!get_code(d, code) || !make_noise(px, py, pz, scale, n)) return -1;
  const int m = (int)code.faces.size();
  if (m > 24) return -1;
  std::vector<uint8_t> C(start, start + code.nq);
  int64_t E = energy(n, C);
  E_out[0] = (int32_t)E;
  const uint64_t total = (uint64_t)1 << m;
  for (uint64_t k = 1; k < total; ++k) {
    int g = __builtin_ctzll(k);
    apply_generator(code, g, C);
    E_out[k] = (int32_t)energy(n, C);
  }
  return 0;
}

}  // extern "C"
