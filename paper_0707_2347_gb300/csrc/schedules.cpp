// The memory schedules of the paper, Tables 1-9, as row lists.
//
// Each row keeps the paper's order and location column.  Values are not
// named here: a row reads the locations the table says hold its operands.
// Readings of ambiguous passages:
//   * Table 6 prints row numbers 5 and 17 twice: rows are taken in printed
//     order (24 rows).
//   * Table 9 row 19 is an AcLR call with alpha and coefficient +1 on C21
//     (holding U2); row 24 is an AccR call with -alpha and coefficient +1 on
//     C21 (holding U3).
//   * The Section 5.1 variant of Table 4 inserts "A21 <- A12" after row 18,
//     "A12 <- A21" after row 19, and calls OvR in row 21.
#include "schedules.h"

namespace swmm {
namespace {

Row ADD(Loc d, Shape sh, Loc a, Coef ca, Loc b, Coef cb) {
  Row r{};
  r.op = OP_ADD;
  r.dst = d;
  r.shape = sh;
  r.s1 = a;
  r.c1 = ca;
  r.s2 = b;
  r.c2 = cb;
  return r;
}
Row MUL(Loc d, Kind k, Coef ca, Loc l, Loc rr) {
  Row r{};
  r.op = OP_MUL;
  r.dst = d;
  r.shape = SH_C;
  r.kind = k;
  r.c1 = ca;
  r.s1 = l;
  r.s2 = rr;
  r.acc = false;
  return r;
}
Row MULACC(Loc d, Kind k, Coef ca, Loc l, Loc rr, Coef cacc) {
  Row r = MUL(d, k, ca, l, rr);
  r.acc = true;
  r.cacc = cacc;
  return r;
}
Row COPY(Loc d, Shape sh, Loc s) {
  Row r{};
  r.op = OP_COPY;
  r.dst = d;
  r.shape = sh;
  r.s1 = s;
  return r;
}

constexpr Coef P = CF_ONE, N = CF_NEG, A = CF_ALPHA, NA = CF_NALPHA, B = CF_BETA, NB = CF_NBETA;

// Table 1: C <- AB with temporaries X, Y (Douglas et al., Section 3.1)
const std::vector<Row> T1 = {
    ADD(LX, SH_A, A11, P, A21, N),   // S3 = A11 - A21
    ADD(LY, SH_B, B22, P, B12, N),   // T3 = B22 - B12
    MUL(C21, K_T1, A, LX, LY),       // P7 = S3 T3
    ADD(LX, SH_A, A21, P, A22, P),   // S1 = A21 + A22
    ADD(LY, SH_B, B12, P, B11, N),   // T1 = B12 - B11
    MUL(C22, K_T1, A, LX, LY),       // P5 = S1 T1
    ADD(LX, SH_A, LX, P, A11, N),    // S2 = S1 - A11
    ADD(LY, SH_B, B22, P, LY, N),    // T2 = B22 - T1
    MUL(C12, K_T1, A, LX, LY),       // P6 = S2 T2
    ADD(LX, SH_A, A12, P, LX, N),    // S4 = A12 - S2
    MUL(C11, K_T1, A, LX, B22),      // P3 = S4 B22
    MUL(LX, K_T1, A, A11, B11),      // P1 = A11 B11
    ADD(C12, SH_C, LX, P, C12, P),   // U2 = P1 + P6
    ADD(C21, SH_C, C12, P, C21, P),  // U3 = U2 + P7
    ADD(C12, SH_C, C12, P, C22, P),  // U4 = U2 + P5
    ADD(C22, SH_C, C21, P, C22, P),  // U7 = U3 + P5
    ADD(C12, SH_C, C12, P, C11, P),  // U5 = U4 + P3
    ADD(LY, SH_B, LY, P, B21, N),    // T4 = T2 - B21
    MUL(C11, K_T1, A, A22, LY),      // P4 = A22 T4
    ADD(C21, SH_C, C21, P, C11, N),  // U6 = U3 - P4
    MUL(C11, K_T1, A, A12, B21),     // P2 = A12 B21
    ADD(C11, SH_C, LX, P, C11, P),   // U1 = P1 + P2
};

// Table 2: C <- aAB + bC with temporaries X, Y, Z (Huss-Lederman et al.)
const std::vector<Row> T2 = {
    ADD(LX, SH_A, A21, P, A22, P),             // S1 = A21 + A22
    ADD(LY, SH_B, B12, P, B11, N),             // T1 = B12 - B11
    MUL(LZ, K_T1, A, LX, LY),                  // P5 = a S1 T1
    ADD(C22, SH_C, LZ, P, C22, B),             // C22 = P5 + b C22
    ADD(C12, SH_C, LZ, P, C12, B),             // C12 = P5 + b C12
    ADD(LX, SH_A, LX, P, A11, N),              // S2 = S1 - A11
    ADD(LY, SH_B, B22, P, LY, N),              // T2 = B22 - T1
    MUL(LZ, K_T1, A, A11, B11),                // P1 = a A11 B11
    ADD(C11, SH_C, LZ, P, C11, B),             // C11 = P1 + b C11
    MULACC(LZ, K_T2, A, LX, LY, P),            // U2 = a S2 T2 + P1
    MULACC(C11, K_T2, A, A12, B21, P),         // U1 = a A12 B21 + C11
    ADD(LX, SH_A, A12, P, LX, N),              // S4 = A12 - S2
    ADD(LY, SH_B, LY, P, B21, N),              // T4 = T2 - B21
    MULACC(C12, K_T2, A, LX, B22, P),          // C12 = a S4 B22 + C12
    ADD(C12, SH_C, LZ, P, C12, P),             // U5 = U2 + C12
    MULACC(C21, K_T2, A, A22, LY, NB),         // P4 = a A22 T4 - b C21
    ADD(LX, SH_A, A11, P, A21, N),             // S3 = A11 - A21
    ADD(LY, SH_B, B22, P, B12, N),             // T3 = B22 - B12
    MULACC(LZ, K_T2, A, LX, LY, P),            // U3 = a S3 T3 + U2
    ADD(C22, SH_C, LZ, P, C22, P),             // U7 = U3 + C22
    ADD(C21, SH_C, LZ, P, C21, N),             // U6 = U3 - C21
};

// Table 3 (IP): C <- AB in place, overwriting A and B (Section 5.1)
const std::vector<Row> T3 = {
    ADD(C11, SH_A, A11, P, A21, N),  // S3 = A11 - A21
    ADD(A21, SH_A, A21, P, A22, P),  // S1 = A21 + A22
    ADD(C22, SH_B, B12, P, B11, N),  // T1 = B12 - B11
    ADD(B12, SH_B, B22, P, B12, N),  // T3 = B22 - B12
    MUL(C21, K_IP, A, C11, B12),     // P7 = IP(S3 T3)
    ADD(C12, SH_A, A21, P, A11, N),  // S2 = S1 - A11
    MUL(C11, K_IP, A, A11, B11),     // P1 = IP(A11 B11)
    ADD(B11, SH_B, B22, P, C22, N),  // T2 = B22 - T1
    MUL(A11, K_IP, A, A21, C22),     // P5 = IP(S1 T1)
    ADD(C22, SH_B, B11, P, B21, N),  // T4 = T2 - B21
    MUL(A21, K_IP, A, A22, C22),     // P4 = IP(A22 T4)
    ADD(A22, SH_A, A12, P, C12, N),  // S4 = A12 - S2
    MUL(C22, K_IP, A, C12, B11),     // P6 = IP(S2 T2)
    ADD(C22, SH_C, C11, P, C22, P),  // U2 = P1 + P6
    MUL(C12, K_IP, A, A12, B21),     // P2 = IP(A12 B21)
    ADD(C11, SH_C, C11, P, C12, P),  // U1 = P1 + P2
    ADD(C12, SH_C, C22, P, A11, P),  // U4 = U2 + P5
    ADD(C22, SH_C, C22, P, C21, P),  // U3 = U2 + P7
    ADD(C21, SH_C, C22, P, A21, N),  // U6 = U3 - P4
    ADD(C22, SH_C, C22, P, A11, P),  // U7 = U3 + P5
    MUL(A12, K_IP, A, A22, B22),     // P3 = IP(S4 B22)
    ADD(C12, SH_C, C12, P, A12, P),  // U5 = U4 + P3
};

// Table 4 (OvL): C <- AB overwriting A, one temporary X
const std::vector<Row> T4 = {
    ADD(C22, SH_A, A11, P, A21, N),  // S3 = A11 - A21
    ADD(A21, SH_A, A21, P, A22, P),  // S1 = A21 + A22
    ADD(C12, SH_A, A21, P, A11, N),  // S2 = S1 - A11
    ADD(C21, SH_B, B12, P, B11, N),  // T1 = B12 - B11
    MUL(C11, K_OVL, A, A11, B11),    // P1 = OvL(A11 B11)
    ADD(A11, SH_B, B22, P, B12, N),  // T3 = B22 - B12
    MUL(LX, K_IP, A, C22, A11),      // P7 = IP(S3 T3)
    ADD(A11, SH_B, B22, P, C21, N),  // T2 = B22 - T1
    MUL(C22, K_IP, A, A21, C21),     // P5 = IP(S1 T1)
    ADD(C21, SH_A, A12, P, C12, N),  // S4 = A12 - S2
    MUL(A21, K_OVL, A, C21, B22),    // P3 = OvL(S4 B22)
    MUL(C21, K_OVL, A, C12, A11),    // P6 = OvL(S2 T2)
    ADD(A11, SH_B, A11, P, B21, N),  // T4 = T2 - B21
    ADD(C21, SH_C, C11, P, C21, P),  // U2 = P1 + P6
    ADD(C12, SH_C, C21, P, C22, P),  // U4 = U2 + P5
    ADD(C21, SH_C, C21, P, LX, P),   // U3 = U2 + P7
    ADD(C22, SH_C, C21, P, C22, P),  // U7 = U3 + P5
    ADD(C12, SH_C, C12, P, A21, P),  // U5 = U4 + P3
    MUL(LX, K_OVL, A, A12, B21),     // P2 = OvL(A12 B21)
    ADD(C11, SH_C, C11, P, LX, P),   // U1 = P1 + P2
    MUL(A21, K_IP, A, A22, A11),     // P4 = IP(A22 T4)
    ADD(C21, SH_C, C21, P, A21, N),  // U6 = U3 - P4
};

// Section 5.1 variant of Table 4 overwriting only A11 and A21
const std::vector<Row> T4M = {
    ADD(C22, SH_A, A11, P, A21, N),  // S3 = A11 - A21
    ADD(A21, SH_A, A21, P, A22, P),  // S1 = A21 + A22
    ADD(C12, SH_A, A21, P, A11, N),  // S2 = S1 - A11
    ADD(C21, SH_B, B12, P, B11, N),  // T1 = B12 - B11
    MUL(C11, K_OVLM, A, A11, B11),   // P1 = OvL(A11 B11)
    ADD(A11, SH_B, B22, P, B12, N),  // T3 = B22 - B12
    MUL(LX, K_IP, A, C22, A11),      // P7 = IP(S3 T3)
    ADD(A11, SH_B, B22, P, C21, N),  // T2 = B22 - T1
    MUL(C22, K_IP, A, A21, C21),     // P5 = IP(S1 T1)
    ADD(C21, SH_A, A12, P, C12, N),  // S4 = A12 - S2
    MUL(A21, K_OVLM, A, C21, B22),   // P3 = OvL(S4 B22)
    MUL(C21, K_OVLM, A, C12, A11),   // P6 = OvL(S2 T2)
    ADD(A11, SH_B, A11, P, B21, N),  // T4 = T2 - B21
    ADD(C21, SH_C, C11, P, C21, P),  // U2 = P1 + P6
    ADD(C12, SH_C, C21, P, C22, P),  // U4 = U2 + P5
    ADD(C21, SH_C, C21, P, LX, P),   // U3 = U2 + P7
    ADD(C22, SH_C, C21, P, C22, P),  // U7 = U3 + P5
    ADD(C12, SH_C, C12, P, A21, P),  // U5 = U4 + P3
    COPY(A21, SH_A, A12),            // 18bis: A21 <- A12
    MUL(LX, K_OVLM, A, A12, B21),    // P2 = OvL(A12 B21)
    COPY(A12, SH_A, A21),            // 19bis: A12 <- A21
    ADD(C11, SH_C, C11, P, LX, P),   // U1 = P1 + P2
    MUL(A21, K_OVR, A, A22, A11),    // P4 = OvR(A22 T4)
    ADD(C21, SH_C, C21, P, A21, N),  // U6 = U3 - P4
};

// Table 5 (OvR): C <- AB overwriting B, one temporary X
const std::vector<Row> T5 = {
    ADD(C22, SH_A, A11, P, A21, N),  // S3 = A11 - A21
    ADD(C21, SH_A, A21, P, A22, P),  // S1 = A21 + A22
    ADD(C12, SH_B, B12, P, B11, N),  // T1 = B12 - B11
    MUL(C11, K_OVR, A, A11, B11),    // P1 = OvR(A11 B11)
    ADD(B11, SH_A, C21, P, A11, N),  // S2 = S1 - A11
    ADD(B12, SH_B, B22, P, B12, N),  // T3 = B22 - B12
    MUL(LX, K_IP, A, C22, B12),      // P7 = IP(S3 T3)
    ADD(B12, SH_B, B22, P, C12, N),  // T2 = B22 - T1
    MUL(C22, K_IP, A, C21, C12),     // P5 = IP(S1 T1)
    ADD(C12, SH_B, B12, P, B21, N),  // T4 = T2 - B21
    MUL(C21, K_OVR, A, B11, B12),    // P6 = OvR(S2 T2)
    MUL(B12, K_OVR, A, A22, C12),    // P4 = OvR(A22 T4)
    ADD(B11, SH_A, A12, P, B11, N),  // S4 = A12 - S2
    ADD(C21, SH_C, C11, P, C21, P),  // U2 = P1 + P6
    ADD(C12, SH_C, C21, P, C22, P),  // U4 = U2 + P5
    ADD(C21, SH_C, C21, P, LX, P),   // U3 = U2 + P7
    ADD(C22, SH_C, C21, P, C22, P),  // U7 = U3 + P5
    ADD(C21, SH_C, C21, P, B12, N),  // U6 = U3 - P4
    MUL(B12, K_IP, A, B11, B22),     // P3 = IP(S4 B22)
    ADD(C12, SH_C, C12, P, B12, P),  // U5 = U4 + P3
    MUL(B12, K_OVR, A, A12, B21),    // P2 = OvR(A12 B21)
    ADD(C11, SH_C, C11, P, B12, P),  // U1 = P1 + P2
};

// Table 6 (AcLR): C <- aAB + bC overwriting A and B, temporaries X, Y
const std::vector<Row> T6 = {
    ADD(C22, SH_C, C22, P, C12, N),       // Z1 = C22 - C12
    ADD(LX, SH_A, A21, P, A22, P),        // S1 = A21 + A22
    ADD(LY, SH_B, B12, P, B11, N),        // T1 = B12 - B11
    ADD(C21, SH_C, C21, P, C22, N),       // Z2 = C21 - Z1
    ADD(B12, SH_B, B22, P, B12, N),       // T3 = B22 - B12
    ADD(A21, SH_A, A11, P, A21, N),       // S3 = A11 - A21
    MULACC(C22, K_ACLR, A, A21, B12, B),  // P7 = AcLR(a S3 T3 + b Z1)
    ADD(A21, SH_A, LX, P, A11, N),        // S2 = S1 - A11
    ADD(B12, SH_B, B22, P, LY, N),        // T2 = B22 - T1
    MULACC(C12, K_ACLR, A, LX, LY, B),    // P5 = AcLR(a S1 T1 + b C12)
    MUL(LY, K_IP, A, A11, B11),           // P1 = a IP(A11 B11)
    ADD(LX, SH_B, B12, P, B21, N),        // T4 = T2 - B21
    MULACC(C21, K_ACLR, A, A22, LX, NB),  // P4 = AcLR(a A22 T4 - b Z2)
    ADD(A22, SH_A, A12, P, A21, N),       // S4 = A12 - S2
    MUL(LX, K_IP, A, A21, B12),           // P6 = a IP(S2 T2)
    MULACC(C11, K_ACLR, A, A12, B21, B),  // P2 = AcLR(a A12 B21 + b C11)
    ADD(C11, SH_C, LY, P, C11, P),        // U1 = P1 + P2
    ADD(LX, SH_C, LY, P, LX, P),          // U2 = P1 + P6
    ADD(C22, SH_C, LX, P, C22, P),        // U3 = U2 + P7
    ADD(LX, SH_C, LX, P, C12, P),         // U4 = U2 + P5
    ADD(C21, SH_C, C22, P, C21, N),       // U6 = U3 - P4
    ADD(C22, SH_C, C22, P, C12, P),       // U7 = U3 + P5
    MUL(C12, K_IP, A, A22, B22),          // P3 = a IP(S4 B22)
    ADD(C12, SH_C, LX, P, C12, P),        // U5 = U4 + P3
};

// Table 7 (AccR): C <- aAB + bC overwriting B, temporaries X, Y
const std::vector<Row> T7 = {
    ADD(C22, SH_C, C22, P, C12, N),       // Z1 = C22 - C12
    ADD(LX, SH_B, B12, P, B11, N),        // T1 = B12 - B11
    ADD(C21, SH_C, C21, P, C22, N),       // Z2 = C21 - Z1
    ADD(B12, SH_B, B22, P, B12, N),       // T3 = B22 - B12
    ADD(LY, SH_A, A11, P, A21, N),        // S3 = A11 - A21
    MULACC(C22, K_ACCR, A, LY, B12, B),   // P7 = AccR(a S3 T3 + b Z1)
    ADD(LY, SH_A, A21, P, A22, P),        // S1 = A21 + A22
    ADD(B12, SH_B, B22, P, LX, N),        // T2 = B22 - T1
    MULACC(C12, K_ACCR, A, LY, LX, B),    // P5 = AccR(a S1 T1 + b C12)
    ADD(LX, SH_B, B12, P, B21, N),        // T4 = T2 - B21
    MULACC(C21, K_ACCR, A, A22, LX, NB),  // P4 = AccR(a A22 T4 - b Z2)
    MUL(LX, K_OVR, A, A11, B11),          // P1 = a OvR(A11 B11)
    MULACC(C11, K_ACCR, A, A12, B21, B),  // P2 = AccR(a A12 B21 + b C11)
    ADD(LY, SH_A, LY, P, A11, N),         // S2 = S1 - A11
    MUL(B21, K_OVR, A, LY, B12),          // P6 = a OvR(S2 T2)
    ADD(LY, SH_A, A12, P, LY, N),         // S4 = A12 - S2
    ADD(B21, SH_C, LX, P, B21, P),        // U2 = P1 + P6
    ADD(C22, SH_C, B21, P, C22, P),       // U3 = U2 + P7
    ADD(B21, SH_C, B21, P, C12, P),       // U4 = U2 + P5
    ADD(C21, SH_C, C22, P, C21, N),       // U6 = U3 - P4
    ADD(C11, SH_C, LX, P, C11, P),        // U1 = P1 + P2
    ADD(C22, SH_C, C22, P, C12, P),       // U7 = U3 + P5
    MUL(C12, K_IP, A, LY, B22),           // P3 = a IP(S4 B22)
    ADD(C12, SH_C, B21, P, C12, P),       // U5 = U4 + P3
};

// Table 8 (AcR): rectangular C <- aAB + bC overwriting B12, B21
const std::vector<Row> T8 = {
    ADD(C22, SH_C, C22, P, C12, N),      // Z1 = C22 - C12
    ADD(LX, SH_B, B12, P, B11, N),       // T1 = B12 - B11
    ADD(C21, SH_C, C21, P, C22, N),      // Z2 = C21 - Z1
    ADD(B12, SH_B, B22, P, B12, N),      // T3 = B22 - B12
    ADD(LY, SH_A, A11, P, A21, N),       // S3 = A11 - A21
    MULACC(C22, K_ACR, A, LY, B12, B),   // P7 = AcR(a S3 T3 + b Z1)
    ADD(LY, SH_A, A21, P, A22, P),       // S1 = A21 + A22
    ADD(B12, SH_B, B22, P, LX, N),       // T2 = B22 - T1
    MULACC(C12, K_ACR, A, LY, LX, B),    // P5 = AcR(a S1 T1 + b C12)
    ADD(LX, SH_B, B12, P, B21, N),       // T4 = T2 - B21
    MULACC(C21, K_ACR, A, A22, LX, NB),  // P4 = AcR(a A22 T4 - b Z2)
    MUL(LX, K_T1, A, A11, B11),          // P1 = a A11 B11
    MULACC(C11, K_ACR, A, A12, B21, B),  // P2 = AcR(a A12 B21 + b C11)
    ADD(C11, SH_C, LX, P, C11, P),       // U1 = P1 + P2
    ADD(LY, SH_A, LY, P, A11, N),        // S2 = S1 - A11
    MULACC(LX, K_ACR, A, LY, B12, P),    // U2 = AcR(a S2 T2 + P1)
    ADD(C22, SH_C, LX, P, C22, P),       // U3 = U2 + P7
    ADD(C21, SH_C, C22, P, C21, N),      // U6 = U3 - P4
    ADD(C22, SH_C, C22, P, C12, P),      // U7 = U3 + P5
    ADD(LX, SH_C, LX, P, C12, P),        // U4 = U2 + P5
    ADD(LY, SH_A, A12, P, LY, N),        // S4 = A12 - S2
    MUL(C12, K_T1, A, LY, B22),          // P3 = a S4 B22
    ADD(C12, SH_C, LX, P, C12, P),       // U5 = U4 + P3
};

// Table 9 (Acc): C <- aAB + bC, read-only A and B, temporaries X, Y
const std::vector<Row> T9 = {
    ADD(C22, SH_C, C22, P, C12, N),        // Z1 = C22 - C12
    ADD(C12, SH_C, C12, P, C21, N),        // Z3 = C12 - C21
    ADD(LX, SH_A, A21, P, A22, P),         // S1 = A21 + A22
    ADD(LY, SH_B, B12, P, B11, N),         // T1 = B12 - B11
    MULACC(C12, K_ACC, A, LX, LY, B),      // P5 = Acc(a S1 T1 + b Z3)
    ADD(LX, SH_A, LX, P, A11, N),          // S2 = S1 - A11
    ADD(LY, SH_B, B22, P, LY, N),          // T2 = B22 - T1
    MULACC(C21, K_ACC, A, LX, LY, B),      // P6 = Acc(a S2 T2 + b C21)
    ADD(LX, SH_A, A12, P, LX, N),          // S4 = A12 - S2
    ADD(C22, SH_C, C12, P, C22, B),        // W1 = P5 + b Z1
    MULACC(C12, K_ACC, A, LX, B22, P),     // P3 = Acc(a S4 B22 + P5)
    MUL(LX, K_T1, A, A11, B11),            // P1 = a A11 B11
    ADD(C21, SH_C, C21, P, LX, P),         // U2 = P6 + P1
    MULACC(C11, K_ACC, A, A12, B21, B),    // P2 = Acc(a A12 B21 + b C11)
    ADD(C11, SH_C, LX, P, C11, P),         // U1 = P1 + P2
    ADD(C12, SH_C, C21, P, C12, P),        // U5 = U2 + P3
    ADD(LX, SH_A, A11, P, A21, N),         // S3 = A11 - A21
    ADD(LY, SH_B, B22, P, B12, N),         // T3 = B22 - B12
    MULACC(C21, K_ACLR, A, LX, LY, P),     // U3 = a AcLR(S3 T3 + U2)
    ADD(C22, SH_C, C21, P, C22, P),        // U7 = U3 + W1
    ADD(LY, SH_B, B12, P, B11, N),         // T1' = B12 - B11
    ADD(LY, SH_B, B22, P, LY, N),          // T2' = B22 - T1'
    ADD(LY, SH_B, LY, P, B21, N),          // T4 = T2' - B21
    MULACC(C21, K_ACCR, NA, A22, LY, P),   // U6 = -a AccR(A22 T4 - U3)
};

const KindInfo kInfo[NKIND] = {
    {"T1", &T1, false, false},  {"T2", &T2, true, false},   {"IP", &T3, false, false},
    {"OvL", &T4, false, true},  {"OvLM", &T4M, false, true}, {"OvR", &T5, false, true},
    {"AcLR", &T6, true, true},  {"AccR", &T7, true, true},  {"AcR", &T8, true, false},
    {"Acc", &T9, true, true},
};

}  // namespace

const KindInfo &kind_info(Kind k) { return kInfo[k]; }

}  // namespace swmm
