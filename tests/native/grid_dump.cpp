// Test harness: builds the library's host grid (grid.cpp) without a GPU and
// writes it as raw little-endian arrays for comparison with the oracle.
// usage: grid_dump refinement n_levels n_r H grading omega2 courant_c centre out.bin
#include <cstdio>
#include <cstdlib>
#include <string>

#include "../../paper_1408_2981_gb300/csrc/tpmg_internal.h"

int main(int argc, char **argv)
{
    if (argc != 10) return 2;
    tpmg_params p{};
    p.refinement = std::atoi(argv[1]);
    p.n_levels = std::atoi(argv[2]);
    p.n_r = std::atoi(argv[3]);
    p.H = std::atof(argv[4]);
    p.grading = std::atof(argv[5]);
    p.omega2 = std::atof(argv[6]);
    p.courant_c = std::atof(argv[7]);
    p.centre = std::atoi(argv[8]);
    tpmg::HostGrid G;
    std::string err;
    if (!tpmg::build_host_grid(p, G, err)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 1;
    }
    FILE *f = std::fopen(argv[9], "wb");
    if (!f) return 3;
    std::fwrite(&G.omega2, sizeof(double), 1, f);
    std::fwrite(&G.h_min, sizeof(double), 1, f);
    std::fwrite(G.r.data(), sizeof(double), G.r.size(), f);
    std::fwrite(G.dr.data(), sizeof(double), G.dr.size(), f);
    std::fwrite(G.vol.data(), sizeof(double), G.vol.size(), f);
    for (int l = p.refinement - p.n_levels + 1; l <= p.refinement; ++l) {
        const tpmg::HostLevel &L = G.lev[l];
        std::fwrite(&L.n, sizeof(int), 1, f);
        std::fwrite(&L.n_colours, sizeof(int), 1, f);
        std::fwrite(L.centre.data(), sizeof(double), L.centre.size(), f);
        std::fwrite(L.area.data(), sizeof(double), L.area.size(), f);
        std::fwrite(L.g.data(), sizeof(double), L.g.size(), f);
        std::fwrite(L.nbr.data(), sizeof(int), L.nbr.size(), f);
        std::fwrite(L.colour.data(), sizeof(int), L.colour.size(), f);
        std::fwrite(L.corner.data(), sizeof(double), L.corner.size(), f);
    }
    std::fclose(f);
    return 0;
}
