"""CPU model of the learned tagger's tensor-core layout (af_cnn.cu, TcGeo and
the two row-shifted GEMMs), restated from the kernel source and walked for
every compiled shape: every operand row an MMA reads lies inside the region
it addresses, every valid output position reads only taps of its own input
row and maps to one layer-1 pixel (or layer-2 pixel), the accumulators fit
the tensor-memory allocation, and four CTAs fit an SM's shared memory (the
occupancy the forward launch assumes).  No GPU needed."""
import pytest

F = 32
SMEM_SM = 233472          # bytes of shared memory per SM (228 KB)
RESERVED = 1024           # per-CTA system reserve
STATIC_FWD = 3456         # static shared memory of the training forward (largest instantiation)


def align128(b):
    return (b + 127) // 128 * 128


def geo(C, N, bwd=False):
    S, S1 = N + 4, N + 2
    g = dict(S=S, S1=S1, P1=S1 * S1, Q1=S1 * S)
    g["MT1"] = (g["Q1"] + 127) // 128
    g["RH"] = g["MT1"] * 128 + 2 * S
    g["Q2"] = N * S1
    g["MT2"] = (g["Q2"] + 127) // 128
    g["R1"] = g["MT2"] * 128 + 2 * S1 + 2
    g["xh_chunk"] = g["RH"] * 16
    g["a1_chunk"] = g["R1"] * 16
    g["xbytes"] = C * S * S * 2
    g["w1t"] = align128((1 if bwd else 2) * g["xbytes"])
    g["w2t"] = g["w1t"] + 3 * 2 * 32 * 16
    g["reg"] = g["w2t"] + (0 if bwd else 9 * 4 * 32 * 16)
    g["reg_bytes"] = 2 * g["xh_chunk"] if bwd else max(2 * g["xh_chunk"], 4 * g["a1_chunk"])
    g["end"] = g["reg"] + g["reg_bytes"]
    return g


@pytest.mark.parametrize("C,N", [(1, 8), (3, 8), (1, 16), (3, 16)])
def test_layer1_shifted_gemms_stay_inside_xh_and_read_their_own_row(C, N):
    g = geo(C, N)
    S, S1 = g["S"], g["S1"]
    assert 3 * C <= 16
    pixels = set()
    for mt in range(g["MT1"]):
        for ky in range(3):
            start = mt * 128 + ky * S                       # A operand start row of this MMA
            assert start + 127 < g["RH"]                    # both 16-byte column blocks hold RH rows
            assert (start * 16) % 16 == 0
        for row in range(128):
            q = mt * 128 + row
            y, x = divmod(q, S)
            if y < S1 and x < S1:                           # a valid layer-1 output
                for ky in range(3):
                    r = q + ky * S                          # Xh row read for tap row ky
                    yy, xx = divmod(r, S)
                    assert yy == y + ky and yy < S
                    for kx in range(3):                     # its taps X[c][r + kx] stay in input row yy
                        assert xx + kx < S and r + kx < S * S
                m = y * S1 + x
                assert 0 <= m < g["P1"] and m not in pixels
                pixels.add(m)
    assert len(pixels) == g["P1"]                           # every layer-1 pixel written once
    assert 32 * g["MT1"] <= 128


@pytest.mark.parametrize("C,N", [(1, 8), (3, 8), (1, 16), (3, 16)])
def test_layer2_shifted_gemms_read_the_map_inside_its_rows(C, N):
    g = geo(C, N)
    S1 = g["S1"]
    outs = set()
    for mt in range(g["MT2"]):
        for sft in range(9):
            ky, kx = divmod(sft, 3)
            start = mt * 128 + ky * S1 + kx
            assert start + 127 < g["R1"]
        for row in range(128):
            q = mt * 128 + row
            y, x = divmod(q, S1)
            if y < N and x < N:                             # a valid layer-2 output: reads written pixels
                for ky in range(3):
                    for kx in range(3):
                        m = q + ky * S1 + kx
                        assert m == (y + ky) * S1 + (x + kx) and m < g["P1"]
                outs.add(y * N + x)
    assert len(outs) == N * N
    assert 32 * g["MT2"] <= 128


@pytest.mark.parametrize("C,N", [(1, 8), (3, 8), (1, 16), (3, 16)])
def test_regions_fit_and_four_ctas_share_an_sm(C, N):
    g = geo(C, N)
    assert g["w1t"] >= 2 * g["xbytes"] and g["w1t"] % 128 == 0
    assert g["reg"] % 16 == 0 and g["xh_chunk"] % 16 == 0 and g["a1_chunk"] % 16 == 0
    assert 2 * g["xh_chunk"] <= g["reg_bytes"] and 4 * g["a1_chunk"] <= g["reg_bytes"]
    assert 4 * (g["end"] + STATIC_FWD + RESERVED) <= SMEM_SM
    b = geo(C, N, bwd=True)
    assert 2 * b["xh_chunk"] == b["reg_bytes"]


def test_model_matches_the_kernels_measured_shared_memory():
    """The model's region sizes are the kernel's: ncu reports 53,376 bytes of
    dynamic shared memory per CTA for cnn_forward_kernel<3, 16, *>."""
    assert geo(3, 16)["end"] == 53376
