// bq_df64.cu -- launches of the double-float hopping kernels (FP64 storage,
// float-pair arithmetic, a lane pair per output site; bq_df64.cuh): single
// system and batched over a unit table, for the storage combinations that the
// operators and solvers use. The intermediate vectors of Mhat and
// Mhat^dag Mhat are float pairs (DF_* flags), the caller's vectors FP64:
//   plain D_hop:           FP64 -> FP64
//   D_oe then A_oo^{-1}:   FP64 -> FP64, FP64 -> pairs, pairs -> pairs
//   A x - k D_eo:          (in, x, out) = (FP64, FP64, FP64), (pairs, FP64, FP64),
//                          (pairs, pairs, FP64), (pairs, FP64, pairs)
#include "bq_internal.cuh"
#include "bq_df64.cuh"

namespace {

template <int EPI>
constexpr bool fmt_ok(int f) {
    return EPI == EPI_PLAIN     ? f == 0
           : EPI == EPI_CLOVINV ? (f == 0 || f == DF_OUT_PAIR || f == (DF_IN_PAIR | DF_OUT_PAIR))
                                : (f == 0 || f == DF_IN_PAIR || f == (DF_IN_PAIR | DF_X_PAIR) ||
                                   f == (DF_IN_PAIR | DF_OUT_PAIR));
}

template <int RECON, bool DAG, int EPI, int F>
bool single_if(int fmt, const DslashArgs &a, unsigned grid, cudaStream_t s) {
    if constexpr (fmt_ok<EPI>(F)) {
        if (fmt == F) {
            k_dslash_df64p<RECON, DAG, EPI, F><<<grid, 128, 0, s>>>(a);
            return true;
        }
    }
    return false;
}

template <int RECON, bool DAG, int EPI, int F>
bool batch_if(int fmt, const DslashBatchTable &tab, const double *mask, int nblocks, cudaStream_t s) {
    if constexpr (fmt_ok<EPI>(F)) {
        if (fmt == F) {
            k_dslash_batch_df64p<RECON, DAG, EPI, F><<<nblocks, 128, 0, s>>>(tab, mask);
            return true;
        }
    }
    return false;
}

template <int RECON, bool DAG, int EPI>
bool single_fmt(int fmt, const DslashArgs &a, unsigned grid, cudaStream_t s) {
    return single_if<RECON, DAG, EPI, 0>(fmt, a, grid, s) || single_if<RECON, DAG, EPI, 1>(fmt, a, grid, s) ||
           single_if<RECON, DAG, EPI, 3>(fmt, a, grid, s) || single_if<RECON, DAG, EPI, 4>(fmt, a, grid, s) ||
           single_if<RECON, DAG, EPI, 5>(fmt, a, grid, s);
}

template <int RECON, bool DAG, int EPI>
bool batch_fmt(int fmt, const DslashBatchTable &tab, const double *mask, int nblocks, cudaStream_t s) {
    return batch_if<RECON, DAG, EPI, 0>(fmt, tab, mask, nblocks, s) || batch_if<RECON, DAG, EPI, 1>(fmt, tab, mask, nblocks, s) ||
           batch_if<RECON, DAG, EPI, 3>(fmt, tab, mask, nblocks, s) || batch_if<RECON, DAG, EPI, 4>(fmt, tab, mask, nblocks, s) ||
           batch_if<RECON, DAG, EPI, 5>(fmt, tab, mask, nblocks, s);
}

template <int RECON>
bool single_r(const DslashArgs &a, bool dag, int epi, unsigned grid, cudaStream_t s) {
    if (dag) {
        if (epi == EPI_PLAIN) return single_fmt<RECON, true, EPI_PLAIN>(a.fmt, a, grid, s);
        if (epi == EPI_CLOVINV) return single_fmt<RECON, true, EPI_CLOVINV>(a.fmt, a, grid, s);
        return single_fmt<RECON, true, EPI_XPAY>(a.fmt, a, grid, s);
    }
    if (epi == EPI_PLAIN) return single_fmt<RECON, false, EPI_PLAIN>(a.fmt, a, grid, s);
    if (epi == EPI_CLOVINV) return single_fmt<RECON, false, EPI_CLOVINV>(a.fmt, a, grid, s);
    return single_fmt<RECON, false, EPI_XPAY>(a.fmt, a, grid, s);
}

template <int RECON>
bool batch_r(const DslashBatchTable &tab, const double *mask, int nblocks, bool dag, int epi, cudaStream_t s) {
    const int fmt = tab.units[0].a.fmt;
    if (dag) {
        if (epi == EPI_PLAIN) return batch_fmt<RECON, true, EPI_PLAIN>(fmt, tab, mask, nblocks, s);
        if (epi == EPI_CLOVINV) return batch_fmt<RECON, true, EPI_CLOVINV>(fmt, tab, mask, nblocks, s);
        return batch_fmt<RECON, true, EPI_XPAY>(fmt, tab, mask, nblocks, s);
    }
    if (epi == EPI_PLAIN) return batch_fmt<RECON, false, EPI_PLAIN>(fmt, tab, mask, nblocks, s);
    if (epi == EPI_CLOVINV) return batch_fmt<RECON, false, EPI_CLOVINV>(fmt, tab, mask, nblocks, s);
    return batch_fmt<RECON, false, EPI_XPAY>(fmt, tab, mask, nblocks, s);
}

}  // namespace

int bq_df64p_launch(int recon, const DslashArgs &a, bool dag, int epi, unsigned grid, cudaStream_t s) {
    const bool ok = recon == 12 ? single_r<12>(a, dag, epi, grid, s) : single_r<18>(a, dag, epi, grid, s);
    if (!ok) {
        bq_set_error("double-float hopping term: no kernel for storage flags %d with epilogue %d", a.fmt, epi);
        return BQ_ERR_ARG;
    }
    return BQ_OK;
}

int bq_df64p_batch_launch(int recon, const DslashBatchTable &tab, const double *mask, int nblocks, bool dag, int epi,
                          cudaStream_t s) {
    if (tab.nunits < 1 || tab.units[0].interleave != 5) {
        bq_set_error("double-float batched hopping term: units must take the lane-pair mapping");
        return BQ_ERR_ARG;
    }
    const bool ok = recon == 12 ? batch_r<12>(tab, mask, nblocks, dag, epi, s)
                                : batch_r<18>(tab, mask, nblocks, dag, epi, s);
    if (!ok) {
        bq_set_error("double-float batched hopping term: no kernel for storage flags %d with epilogue %d",
                     tab.units[0].a.fmt, epi);
        return BQ_ERR_ARG;
    }
    return BQ_OK;
}
