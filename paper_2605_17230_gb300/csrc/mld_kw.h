// Kac-Ward planar solver for independent X/Z noise (Sec. 3.1.3): the spin
// graph of one part (X-type plaquettes, the qubits as edges, two ghost
// vertices for the boundary qubits and a tie edge between the ghosts that
// selects the logical sector), its straight-line embedding, and the matrix
// I - Lambda over directed edges in the order the device elimination uses.
#pragma once

#include <stdint.h>

#include <vector>

namespace mld {

struct KwGraph {
    int d = 0;
    int N = 0;        // directed edges = matrix order
    int Nb = 0;       // band part: rows/columns 0..Nb-1; Nb, Nb+1 are the border (the tie's middle edge)
    int bl = 0, bu = 0;   // lower / upper bandwidth of the band part
    int n_plaq = 0;   // spins that are plaquettes (the constant (n_plaq - n) ln 2)
    // I - Lambda in CSR, rows and columns in elimination order, diagonal not
    // stored: entry value = -w(src) * phase. src >= 0: the qubit of the
    // column's edge (index on the lattice whose X-type plaquettes are the
    // vertices); -1: weight 1 (a bend or tie segment); -2: the sector edge
    // (weight +1 in sector 0, -1 in sector 1). The sector edge's two directed
    // edges are columns Nb-2 and Nb-1.
    std::vector<int> row_start, col, src;
    std::vector<double> ph_re, ph_im;
    std::vector<int> ext0;    // per band row: its largest band column (diagonal included)
};

// Builds the graph of the rotated code of distance d (odd, >= 3). Returns
// false if an internal check fails (it does not for odd d >= 3).
bool build_kw_graph(int d, KwGraph* g);

// The Z part is the X part of the lattice turned by a quarter: qubit (r, c)
// of the turned lattice is qubit (d-1-c, r) of the code. zmap[q'] = q.
std::vector<int> kw_zmap(int d);

}  // namespace mld
