"""The oracle and the CUDA path keep separate copies of every constant of the
readings (they share no code); this checks, from the sources as text, that
the copies agree, so that a change on one side cannot pass unnoticed on a
machine without a GPU."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def src(*p):
    return open(os.path.join(ROOT, *p)).read()


def c_define(text, name):
    m = re.search(r"#define\s+%s\s+([0-9.eE+-]+)" % name, text)
    assert m, name
    return float(m.group(1))


def cu_const(text, name):
    m = re.search(r"constexpr\s+\w+(?:\s+\w+)?\s+%s\s*=\s*([0-9.eE+-]+)f?\s*;" % name, text)
    assert m, name
    return float(m.group(1).rstrip("f"))


def test_continuous_readout_constants():
    o = src("oracle", "o2tpc_oracle.c")
    k = src("paper_2106_03636_gb300", "csrc", "k_cont.cu")
    pairs = [("O_SIGMA_ZV", "kSigmaZv"), ("O_MEM_ROWGAP", "kMemRowGap"), ("O_MEM_DZU", "kMemDZetaUnits"),
             ("O_CHI2_MEM", "kChi2Mem"), ("O_MEM_ZTOL", "kMemZTol"), ("O_T0_SLACK", "kT0Slack")]
    for a, b in pairs:
        assert c_define(o, a) == cu_const(k, b), (a, b)


def test_compressed_tf_constants():
    o = src("oracle", "o2tpc_ctf.c")
    k = src("paper_2106_03636_gb300", "csrc", "k_ctf.cu")
    h = src("paper_2106_03636_gb300", "csrc", "o2tpc_ctf_host.cu")
    assert c_define(o, "C_SCALE_BITS") == cu_const(k, "kCtfScaleBits") == 12
    assert c_define(o, "C_CHUNK") == cu_const(k, "kCtfChunk") == 4096
    assert c_define(o, "C_NSTREAM") == cu_const(k, "kCtfStreams") == 10
    # removal of tracks with |q/pT| > 10 / GeV (the oracle states it in code)
    assert cu_const(k, "kCtfMaxQpt") == 10.0
    assert "trk_qpt[t] >= -10.0 && trk_qpt[t] <= 10.0" in o
    assert cu_const(h, "kChunk") == 4096 and cu_const(h, "kStreams") == 10
    assert "kScaleBits = 12" in h and "kL = 1u << 23" in h and "(1u << 23)" in o


def test_clusterizer_constants():
    o = src("oracle", "o2tpc_clu.c")
    k = src("paper_2106_03636_gb300", "csrc", "k_clu.cu")
    assert c_define(o, "U_PEAK_MIN") == cu_const(k, "kPeakMin") == 3


def test_tracking_constants():
    o = src("oracle", "o2tpc_oracle.c")
    k = src("paper_2106_03636_gb300", "csrc", "o2tpc_internal.cuh")
    pairs = [("O_CY", "kCellY"), ("O_T", "kHitsPerCell"), ("O_WY", "kWinY"), ("O_WZ", "kWinZ"),
             ("O_SY", "kSigY"), ("O_SZ", "kSigZ"), ("O_G", "kMaxMiss"), ("O_NMIN", "kMinHits"),
             ("O_CHI2_FOLLOW", "kChi2Follow"), ("O_SIN_FOLLOW", "kSinFollow"), ("O_SIN_PROP", "kSinProp"),
             ("O_EDGE", "kEdgeBand"), ("O_DZETA_PRE", "kMergeDZeta"), ("O_CHI2_MERGE", "kChi2Merge")]
    for a, b in pairs:
        assert c_define(o, a) == cu_const(k, b), (a, b)
    # the integer metric: weights and cut
    assert re.search(r"#define O_AY 2077LL", o) and cu_const(k, "kWeightY") == 2077
    assert re.search(r"#define O_AZ 1536LL", o) and cu_const(k, "kWeightZ") == 1536
    assert "#define O_DMAX (16LL * 1536LL * 2077LL)" in o and "kMaxMetric = 16 * 1536 * 2077;" in k
