/*
 * Plain CPU oracle for the GPS L1 C/A tracking-loop software correlator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library (the CUDA path
 * behind include/rx.h) includes, links or calls this file; only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark do.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * What it computes, and where that is defined:
 *   - the C/A ranging code of Sec. 3.1 (1023 chips, 1.023 Mcps, one code per
 *     SV 1..32).  The paper gives only these properties; the generator
 *     polynomials and the per-PRN G2 phase-selector taps are those of the
 *     public GPS interface specification IS-GPS-200, Table 3-Ia.
 *   - the carrier wipe-off and code-phase alignment of Sec. 3.1 (Fig. 7), in
 *     a fixed-point form: a 32-bit carrier phase accumulator whose top 6 bits
 *     index a 64-entry int8 cos/sin table; a 32.32 fixed-point code phase in
 *     chips; int8 I/Q samples; int32 integrate-and-dump accumulators with
 *     two's-complement wrap (Sec. 4: 1 ms integration).
 *   - the tracking loops of Table 3: normalised early-minus-late envelope
 *     DLL discriminator with carrier aiding, atan PLL discriminator, a
 *     2nd-order PLL and a 1st-order DLL, followed by re-quantisation of the
 *     NCO words; and Table 3's full set (2nd-order PLL with a 1st-order atan2
 *     FLL assist, 2nd-order DLL) with Sec. 4's channel-health indicators
 *     (C/N0, carrier lock ratio, lock-fail count).
 *   - the acquisition search of Sec. 3.3 / 3.6 / 3.7: for each PRN, the power
 *     of the circular correlation of the carrier-wiped buffer with the local
 *     code over a grid of Doppler bins and all code delays (the quantity a
 *     parallel-code-phase FFT search computes), its peak, the second peak of
 *     the peak's Doppler row, and the hand-over of the result to tracking.
 *   - tracking in code-period epochs (one dump per period of each channel's
 *     own prompt code, of varying sample count) and bit synchronisation by a
 *     histogram of prompt sign changes over the 20 code periods of a bit
 *     (Sec. 3.1), with the decoded bits.
 *   Every floating-point step is a single correctly rounded
 *     IEEE-754 binary64 operation, written one per statement, in a fixed
 *     order; the file must be compiled with -ffp-contract=off.
 *
 * Everything is written the slow, literal way: each sample recomputes its
 * carrier and code phase from the block start, every modulo is explicit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CODE_LEN 1023
/* one code period in 32.32 fixed-point chips */
#define ORC_CODE_MOD ((uint64_t)ORC_CODE_LEN << 32)

/* ------------------------------------------------------------------------ */
/* C/A code (Sec. 3.1; generator per IS-GPS-200 Sec. 3.3.2.3, Table 3-Ia)    */
/* ------------------------------------------------------------------------ */

/* G2 phase-selector tap pairs, PRN 1..32 (IS-GPS-200 Table 3-Ia). */
static const int orc_g2_select[32][2] = {
    {2, 6},  {3, 7},  {4, 8},  {5, 9},  {1, 9},  {2, 10}, {1, 8},  {2, 9},
    {3, 10}, {2, 3},  {3, 4},  {5, 6},  {6, 7},  {7, 8},  {8, 9},  {9, 10},
    {1, 4},  {2, 5},  {3, 6},  {4, 7},  {5, 8},  {6, 9},  {1, 3},  {4, 6},
    {5, 7},  {6, 8},  {7, 9},  {8, 10}, {1, 6},  {2, 7},  {3, 8},  {4, 9}};

/*
 * Logic-level chips (0/1) of the C/A code of one PRN, by the two 10-stage
 * shift registers: G1 = 1 + x^3 + x^10, G2 = 1 + x^2 + x^3 + x^6 + x^8 +
 * x^9 + x^10, both preset to all ones; the chip is G1's last stage XOR the
 * XOR of the two G2 stages selected for the PRN.
 */
int orc_ca_logic(int prn, uint8_t out[ORC_CODE_LEN]) {
    if (prn < 1 || prn > 32) return -1;
    int g1[11], g2[11];
    for (int i = 1; i <= 10; ++i) { g1[i] = 1; g2[i] = 1; }
    int a = orc_g2_select[prn - 1][0], b = orc_g2_select[prn - 1][1];
    for (int n = 0; n < ORC_CODE_LEN; ++n) {
        int g2i = g2[a] ^ g2[b];
        out[n] = (uint8_t)(g1[10] ^ g2i);
        int f1 = g1[3] ^ g1[10];
        int f2 = g2[2] ^ g2[3] ^ g2[6] ^ g2[8] ^ g2[9] ^ g2[10];
        for (int i = 10; i >= 2; --i) { g1[i] = g1[i - 1]; g2[i] = g2[i - 1]; }
        g1[1] = f1;
        g2[1] = f2;
    }
    return 0;
}

/*
 * The same code by the equivalent "G2 delay" description: the chip at index n
 * is G1(n) XOR G2(n - D) with D the PRN's code delay in chips.  The delays
 * are passed in by the caller (tests take them from the specification's
 * table) so that the two descriptions can be checked against each other.
 */
int orc_ca_logic_delay(int delay, uint8_t out[ORC_CODE_LEN]) {
    uint8_t g1s[ORC_CODE_LEN], g2s[ORC_CODE_LEN];
    int g1[11], g2[11];
    for (int i = 1; i <= 10; ++i) { g1[i] = 1; g2[i] = 1; }
    for (int n = 0; n < ORC_CODE_LEN; ++n) {
        g1s[n] = (uint8_t)g1[10];
        g2s[n] = (uint8_t)g2[10];
        int f1 = g1[3] ^ g1[10];
        int f2 = g2[2] ^ g2[3] ^ g2[6] ^ g2[8] ^ g2[9] ^ g2[10];
        for (int i = 10; i >= 2; --i) { g1[i] = g1[i - 1]; g2[i] = g2[i - 1]; }
        g1[1] = f1;
        g2[1] = f2;
    }
    for (int n = 0; n < ORC_CODE_LEN; ++n) {
        int m = ((n - delay) % ORC_CODE_LEN + ORC_CODE_LEN) % ORC_CODE_LEN;
        out[n] = (uint8_t)(g1s[n] ^ g2s[m]);
    }
    return 0;
}

/* Bipolar chips: logic 0 -> +1, logic 1 -> -1. */
int orc_ca_code(int prn, int8_t out[ORC_CODE_LEN]) {
    uint8_t logic[ORC_CODE_LEN];
    if (orc_ca_logic(prn, logic) != 0) return -1;
    for (int n = 0; n < ORC_CODE_LEN; ++n) out[n] = logic[n] ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Carrier NCO table (Sec. 3.1 carrier wipe-off)                             */
/* ------------------------------------------------------------------------ */

/* Entry k holds round(127 cos(2 pi k / 64)), round(127 sin(2 pi k / 64)):
 * phase taken at the start of the bin, rounding half away from zero. */
void orc_sincos_table(int8_t cos_tab[64], int8_t sin_tab[64]) {
    for (int k = 0; k < 64; ++k) {
        double ang = 2.0 * M_PI * (double)k / 64.0;
        cos_tab[k] = (int8_t)lround(127.0 * cos(ang));
        sin_tab[k] = (int8_t)lround(127.0 * sin(ang));
    }
}

/* ------------------------------------------------------------------------ */
/* Correlator: carrier wipe-off, code wipe-off at each tap, integrate        */
/* ------------------------------------------------------------------------ */

/*
 * One block of nsamp complex samples for one channel.  For sample n:
 *   theta_n = theta0 + n*w                     (mod 2^32)
 *   (c, s)  = TAB[theta_n >> 26]
 *   I' = I c + Q s,  Q' = Q c - I s            (multiply by exp(-j theta))
 *   phi_n   = phi0 + n*r                       (mod 1023 * 2^32)
 *   chip_k  = ((phi_n + off_k) mod 1023*2^32) >> 32
 *   A_I[k] += code[chip_k] I',  A_Q[k] += code[chip_k] Q'   (mod 2^32)
 * and at the end theta0 += nsamp*w, phi0 = (phi0 + nsamp*r) mod 1023*2^32.
 * acc is [ntaps][2] = {A_I, A_Q}, accumulated into (not cleared).
 */
void orc_correlate_block(const int8_t *iq, uint32_t nsamp, uint32_t *theta0,
                         int32_t w, uint64_t *phi0, uint64_t r,
                         const int64_t *tap_off, uint32_t ntaps,
                         const int8_t code[ORC_CODE_LEN], int32_t *acc) {
    int8_t ctab[64], stab[64];
    orc_sincos_table(ctab, stab);
    uint32_t *uacc = (uint32_t *)acc;
    for (uint32_t n = 0; n < nsamp; ++n) {
        uint32_t theta = *theta0 + n * (uint32_t)w;
        uint32_t k = theta >> 26;
        int32_t c = ctab[k], s = stab[k];
        int32_t I = iq[2 * (size_t)n], Q = iq[2 * (size_t)n + 1];
        int32_t Ip = I * c + Q * s;
        int32_t Qp = Q * c - I * s;
        unsigned __int128 ph = ((unsigned __int128)*phi0 +
                                (unsigned __int128)n * r) % ORC_CODE_MOD;
        for (uint32_t t = 0; t < ntaps; ++t) {
            __int128 x = ((__int128)ph + tap_off[t]) % (__int128)ORC_CODE_MOD;
            if (x < 0) x += ORC_CODE_MOD;
            uint32_t chip = (uint32_t)((uint64_t)x >> 32);
            int32_t g = code[chip];
            uacc[2 * t] += (uint32_t)(g * Ip);
            uacc[2 * t + 1] += (uint32_t)(g * Qp);
        }
    }
    *theta0 = *theta0 + nsamp * (uint32_t)w;
    *phi0 = (uint64_t)(((unsigned __int128)*phi0 +
                        (unsigned __int128)nsamp * r) % ORC_CODE_MOD);
}

/* ------------------------------------------------------------------------ */
/* Arctangent of a ratio, in cycles (PLL discriminator, Table 3)            */
/* ------------------------------------------------------------------------ */

#define ORC_SQRT2 1.4142135623730951
#define ORC_KAID 0.0006493506493506494 /* 1 / 1540 = 1.023e6 / 1575.42e6 */
#define ORC_TWO_M32 2.3283064365386963e-10 /* 2^-32, exact */

/* Breakpoints c_k = tan(k pi/256), k = 0..64 (correctly rounded). */
static const double orc_tan_k[65] = {
    0.0, 0.012272462379566276, 0.024548622108925444, 0.03683218099484564,
    0.049126849769467254, 0.061436352581593766, 0.07376443152244928, 0.0861148511976279,
    0.09849140335716425, 0.11089791159591303, 0.12333823613673868, 0.13581627870938773,
    0.14833598753834742, 0.16090136245348916, 0.17351646013785577, 0.18618539952758373,
    0.198912367379658, 0.21170162402398335, 0.2245575093171293, 0.23748444881607017,
    0.25048696019130545, 0.263569659899918, 0.2767372701404143, 0.2899946261126061,
    0.3033466836073424, 0.3167985269526038, 0.3303553773443339, 0.3440226015924263,
    0.3578057213145241, 0.37171042261274345, 0.38574256627112125, 0.3999081985145372,
    0.41421356237309503, 0.4286651096994995, 0.44326951389086433, 0.4580336833706724,
    0.4729647758913199, 0.48807021372286286, 0.5033576997992942, 0.5188352348999757,
    0.5345111359507917, 0.5503940555372641, 0.566493002730344, 0.5828173653349761,
    0.5993769336819238, 0.6161819260948661, 0.6332430161775692, 0.6505713620801533,
    0.6681786379192989, 0.6860770675448629, 0.7042794608650442, 0.7227992529642059,
    0.7416505462720354, 0.7608481560702512, 0.7804076596539437, 0.8003454494993201,
    0.8206787908286604, 0.8414258840072548, 0.8626059322567399, 0.8842392152253499,
    0.9063471690191471, 0.9289524733703675, 0.9520791467009253, 0.9757526499323765,
    1.0,
};
/* Single-precision midpoints tan((j + 1/2) pi/256), j = 0..63, that choose k. */
static const float orc_mid_k[64] = {
    0.006136000156402588f, 0.0184098482131958f, 0.030689245089888573f, 0.042977895587682724f,
    0.05527951195836067f, 0.06759783625602722f, 0.07993661612272263f, 0.09229962527751923f,
    0.10469067096710205f, 0.11711360514163971f, 0.1295723021030426f, 0.1420706808567047f,
    0.1546127200126648f, 0.1672024428844452f, 0.179843932390213f, 0.19254136085510254f,
    0.20529894530773163f, 0.21812096238136292f, 0.23101182281970978f, 0.24397596716880798f,
    0.25701799988746643f, 0.2701425552368164f, 0.28335443139076233f, 0.2966585159301758f,
    0.3100598156452179f, 0.32356348633766174f, 0.3371748626232147f, 0.3508993089199066f,
    0.3647425174713135f, 0.37871018052101135f, 0.39280831813812256f, 0.4070430099964142f,
    0.4214206635951996f, 0.4359477758407593f, 0.45063120126724243f, 0.46547791361808777f,
    0.4804952144622803f, 0.4956907033920288f, 0.5110722184181213f, 0.5266478657722473f,
    0.5424261689186096f, 0.558415949344635f, 0.5746263861656189f, 0.5910671353340149f,
    0.6077480912208557f, 0.6246797442436218f, 0.6418730616569519f, 0.6593393683433533f,
    0.6770906448364258f, 0.695139467716217f, 0.7134988307952881f, 0.7321825623512268f,
    0.7512050867080688f, 0.7705816626548767f, 0.7903282046318054f, 0.8104615807533264f,
    0.8309994339942932f, 0.8519605398178101f, 0.8733646273612976f, 0.8952324986457825f,
    0.9175862073898315f, 0.940449059009552f, 0.9638459086418152f, 0.9878028631210327f,
};
/* Gregory coefficients divided by 2 pi: (-1)^j / ((2j + 1) 2 pi), j = 0..4. */
static const double orc_series[5] = {0.15915494309189535, -0.05305164769729845, 0.03183098861837907,
                                     -0.022736420441699334, 0.017683882565766147};

/*
 * atan(q / i) / (2 pi), in cycles, for i != 0 (two-quadrant), by table-driven
 * argument reduction:
 *   a = |q|, b = |i|; if a > b swap them and use atan(x) = pi/2 - atan(1/x);
 *   k = the number of midpoints at or below a/b (single-precision estimate of
 *   a/b, binary search), so that c_k = tan(k pi/256) is the breakpoint nearest
 *   a/b (or a neighbour of it);
 *   atan(a/b) = k pi/256 + atan(t),  t = (a - c_k b) / (b + c_k a),  |t| < 0.019;
 *   atan(t) / (2 pi) = t (D0 + D1 u + D2 u^2 + D3 u^3 + D4 u^4), u = t^2, the
 *   Gregory series to t^9 (truncation below t^10 / 11 < 4e-19 relative),
 *   evaluated by Estrin's scheme: (D0 + D1 u) + u^2 ((D2 + D3 u) + u^2 D4);
 *   k pi/256 is k / 512 cycles and pi/2 is 1/4 cycle, both exact.
 * The sign is that of q / i.  One division.
 */
double orc_atan_cycles(double q, double i) {
    double a = fabs(q), b = fabs(i);
    int swap = a > b;
    if (swap) {
        double tmp = a;
        a = b;
        b = tmp;
    }
    float rf = (float)a / (float)b;
    int k = 0;
    for (int step = 32; step >= 1; step >>= 1)
        if (rf >= orc_mid_k[k + step - 1]) k += step;
    double c = orc_tan_k[k];
    double num = c * b;
    num = a - num;
    double den = c * a;
    den = b + den;
    double t = num / den;
    double u = t * t;
    double u2 = u * u;
    double p01 = orc_series[1] * u;
    p01 = orc_series[0] + p01;
    double p23 = orc_series[3] * u;
    p23 = orc_series[2] + p23;
    double p4 = orc_series[4] * u2;
    double hi = p23 + p4;
    hi = hi * u2;
    double p = p01 + hi;
    double y = t * p;
    y = (double)k / 512.0 + y;
    if (swap) y = 0.25 - y;
    if ((q < 0.0) != (i < 0.0)) y = -y;
    return y;
}

/* ------------------------------------------------------------------------ */
/* Tracking loops (Table 3) and NCO re-quantisation                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t theta;   /* carrier phase, 2^-32 cycles */
    int32_t w;        /* carrier phase increment per sample */
    uint64_t phi;     /* code phase, 32.32 chips, in [0, 1023*2^32) */
    uint64_t r;       /* code phase increment per sample, 32.32 chips */
    double v;         /* PLL integrator, Hz */
    double f_carr;    /* last carrier frequency from the PLL, Hz */
    double f_code;    /* last code rate from the DLL, chips/s */
} orc_chan;

/* Initial loop state from the NCO words: the PLL integrator starts at the
 * carrier frequency the word represents. */
void orc_chan_init(orc_chan *ch, int32_t w, uint64_t phi, uint64_t r, double fs) {
    ch->theta = 0;
    ch->w = w;
    ch->phi = phi % ORC_CODE_MOD;
    ch->r = r;
    double f = (double)w * fs;
    ch->v = f / 4294967296.0;
    ch->f_carr = ch->v;
    double fc = (double)r * fs;
    ch->f_code = fc / 4294967296.0;
}

/*
 * One loop update at an integration boundary.  acc = [ntaps][2] dumped sums,
 * n_accum = samples integrated.  Discriminators (Table 3):
 *   PLL: e_p = atan(Q_P / I_P) / (2 pi)           cycles (two-quadrant)
 *   DLL: e_c = (1 - d/2) (|E| - |L|) / (|E| + |L|) chips, d = E-L spacing
 * Filters, with T = n_accum / fs and w0 = Bn_pll / 0.53:
 *   v      = v + (w0^2 T) e_p
 *   f_carr = v + (sqrt2 w0) e_p
 *   f_code = 1.023e6 (1 + f_carr / 1575.42e6) + (4 Bn_dll) e_c   (carrier aided)
 * Re-quantisation, round half to even, with s = 2^32 / fs:
 *   w = rn(f_carr s) (wrapped to int32), r = rn(f_code s)
 * The carrier aiding is evaluated as 1.023e6 + f_carr / 1540 (1575.42 / 1.023
 * = 1540), the division by a multiplication with the correctly rounded 1/1540.
 */
void orc_track(orc_chan *ch, const int32_t *acc, const int64_t *tap_off,
               int tap_e, int tap_p, int tap_l, double fs, uint64_t n_accum,
               double pll_bn, double dll_bn) {
    double T = (double)n_accum / fs;
    double w0 = pll_bn / 0.53;
    double k1 = w0 * w0;
    k1 = k1 * T;
    double k2 = ORC_SQRT2 * w0;
    double kdll = 4.0 * dll_bn;
    double sfs = 4294967296.0 / fs;

    double ip = (double)acc[2 * tap_p], qp = (double)acc[2 * tap_p + 1];
    double e_pll;
    if (ip != 0.0) {
        e_pll = orc_atan_cycles(qp, ip);
    } else {
        e_pll = qp > 0.0 ? 0.25 : (qp < 0.0 ? -0.25 : 0.0);
    }
    double dv = k1 * e_pll;
    ch->v = ch->v + dv;
    double df = k2 * e_pll;
    double f_carr = ch->v + df;

    double ie = (double)acc[2 * tap_e], qe = (double)acc[2 * tap_e + 1];
    double il = (double)acc[2 * tap_l], ql = (double)acc[2 * tap_l + 1];
    double ie2 = ie * ie, qe2 = qe * qe, il2 = il * il, ql2 = ql * ql;
    double mag_e = sqrt(ie2 + qe2);
    double mag_l = sqrt(il2 + ql2);
    double den = mag_e + mag_l;
    double d_el = (double)(tap_off[tap_e] - tap_off[tap_l]) * ORC_TWO_M32;
    double kd = d_el * 0.5;
    kd = 1.0 - kd;
    double e_dll = 0.0;
    if (den > 0.0) {
        double num = mag_e - mag_l;
        num = kd * num;
        e_dll = num / den;
    }
    double aid = f_carr * ORC_KAID;
    double corr = kdll * e_dll;
    double f_code = 1.023e6 + aid;
    f_code = f_code + corr;

    double xw = f_carr * sfs;
    double xr = f_code * sfs;
    /* words: carrier wraps modulo 2^32, code rate clamped to [0, 2^32 - 1] (the range set-up accepts) */
    if (xw > 9.0e18) xw = 9.0e18;
    if (xw < -9.0e18) xw = -9.0e18;
    if (!(xr > 0.0)) xr = 0.0;
    if (xr > 4294967295.0) xr = 4294967295.0;
    ch->w = (int32_t)(uint32_t)(uint64_t)(int64_t)nearbyint(xw);
    ch->r = (uint64_t)nearbyint(xr);
    ch->f_carr = f_carr;
    ch->f_code = f_code;
}

/* ------------------------------------------------------------------------ */
/* Table 3's full loop set and the channel-health indicators of Sec. 4       */
/* ------------------------------------------------------------------------ */

/*
 * atan2(y, x) / (2 pi) in cycles, four quadrants, in (-1/2, 1/2]: the FLL's
 * discriminator (Table 3: FLL atan2).  Built on orc_atan_cycles (two
 * quadrants) by the quadrant of (x, y); +-1/2 cycle is exact.
 */
double orc_atan2_cycles(double y, double x) {
    if (x == 0.0) return y > 0.0 ? 0.25 : (y < 0.0 ? -0.25 : 0.0);
    double a = orc_atan_cycles(y, x);
    if (x > 0.0) return a;
    if (y >= 0.0) return a + 0.5;
    return a - 0.5;
}

/* Extra per-channel state of the full loop set and the health indicators. */
typedef struct {
    int32_t prev_ip, prev_qp;  /* the previous integration's prompt (FLL) */
    uint32_t have_prev;        /* 1 once a previous prompt exists */
    uint32_t window_count;     /* integrations in the current health window */
    double dll_u;              /* 2nd-order DLL's rate integrator, chips/s */
    double sum_abs_ip;         /* window sums: |I_P| */
    double sum_power;          /*   I_P^2 + Q_P^2 */
    double sum_diff;           /*   I_P^2 - Q_P^2 */
    double cn0_hz;             /* last C/N0, linear (Hz); 0 before the first window */
    double lock_ratio;         /* last carrier lock ratio (cos of twice the phase error) */
    uint32_t lock_fail;        /* windows whose lock ratio was below 0.85 */
    uint32_t pad;
} orc_ext;

void orc_ext_init(orc_ext *ex) { memset(ex, 0, sizeof *ex); }

/*
 * One update of Table 3's full loop set at an integration boundary (T =
 * n_accum / fs):
 *   PLL discriminator   e_p = atan(Q_P / I_P) / (2 pi)                 cycles
 *   FLL discriminator   e_f = atan2(s cross, s dot) / (2 pi) / T       Hz
 *                       cross = I1 Q2 - I2 Q1, dot = I1 I2 + Q1 Q2 (1 = previous,
 *                       2 = this integration's prompt; e_f = 0 without a previous one),
 *                       s = sign(dot): the decision on the product of the two data bits,
 *                       removed so that a bit change does not read as a frequency error
 *   carrier filter      2nd-order PLL with 1st-order FLL assist, w0p = Bn_pll / 0.53,
 *                       w0f = 4 Bn_fll:
 *                         v      = v + (w0p^2 T) e_p + (w0f T) e_f
 *                         f_carr = v + (sqrt2 w0p) e_p
 *   DLL discriminator   e_c as in orc_track (normalised E-L envelope)
 *   code filter         2nd-order DLL, carrier aided, w0d = Bn_dll / 0.53:
 *                         u      = u + (w0d^2 T) e_c
 *                         f_code = 1.023e6 + f_carr / 1540 + (u + (sqrt2 w0d) e_c)
 * and the words as in orc_track.  Health (Sec. 4's channel-health indicators),
 * over windows of `window` integrations: C/N0 by the signal-to-noise-variance
 * estimator, Pd = (mean |I_P|)^2, Pn = mean(I_P^2 + Q_P^2) - Pd, C/N0 = Pd / Pn / T
 * (linear, Hz; 0 if Pn <= 0); carrier lock ratio sum(I_P^2 - Q_P^2) / sum(I_P^2 +
 * Q_P^2), the estimate of cos(2 x phase error); the lock-fail count grows by one for
 * each window whose ratio is below 0.85.  One IEEE op per statement, in order.
 */
void orc_track_table3(orc_chan *ch, orc_ext *ex, const int32_t *acc, const int64_t *tap_off,
                      int tap_e, int tap_p, int tap_l, double fs, uint64_t n_accum,
                      double pll_bn, double dll_bn, double fll_bn, uint32_t window) {
    double T = (double)n_accum / fs;
    double inv_T = fs / (double)n_accum;
    double w0p = pll_bn / 0.53;
    double k1 = w0p * w0p;
    k1 = k1 * T;
    double k2 = ORC_SQRT2 * w0p;
    double kf = 4.0 * fll_bn;
    kf = kf * T;
    double w0d = dll_bn / 0.53;
    double kd1 = w0d * w0d;
    kd1 = kd1 * T;
    double kd2 = ORC_SQRT2 * w0d;
    double sfs = 4294967296.0 / fs;

    int32_t ipi = acc[2 * tap_p], qpi = acc[2 * tap_p + 1];
    double ip = (double)ipi, qp = (double)qpi;
    double e_p;
    if (ip != 0.0) {
        e_p = orc_atan_cycles(qp, ip);
    } else {
        e_p = qp > 0.0 ? 0.25 : (qp < 0.0 ? -0.25 : 0.0);
    }
    double e_f = 0.0;
    if (ex->have_prev) {
        double i1 = (double)ex->prev_ip, q1 = (double)ex->prev_qp;
        double a = i1 * qp;
        double b = ip * q1;
        double cross = a - b;
        double c = i1 * ip;
        double d = q1 * qp;
        double dot = c + d;
        /* a data-bit change between the two integrations turns the prompt by half a
         * cycle; the product of the two bits is taken as sign(dot) and removed */
        if (dot < 0.0) {
            cross = -cross;
            dot = -dot;
        }
        double ef = orc_atan2_cycles(cross, dot);
        e_f = ef * inv_T;
    }
    double dv = k1 * e_p;
    double dvf = kf * e_f;
    double v = ch->v + dv;
    v = v + dvf;
    ch->v = v;
    double df = k2 * e_p;
    double f_carr = v + df;

    double ie = (double)acc[2 * tap_e], qe = (double)acc[2 * tap_e + 1];
    double il = (double)acc[2 * tap_l], ql = (double)acc[2 * tap_l + 1];
    double ie2 = ie * ie, qe2 = qe * qe, il2 = il * il, ql2 = ql * ql;
    double mag_e = sqrt(ie2 + qe2);
    double mag_l = sqrt(il2 + ql2);
    double den = mag_e + mag_l;
    double d_el = (double)(tap_off[tap_e] - tap_off[tap_l]) * ORC_TWO_M32;
    double kd = d_el * 0.5;
    kd = 1.0 - kd;
    double e_c = 0.0;
    if (den > 0.0) {
        double num = mag_e - mag_l;
        num = kd * num;
        e_c = num / den;
    }
    double du = kd1 * e_c;
    double u = ex->dll_u + du;
    ex->dll_u = u;
    double aid = f_carr * ORC_KAID;
    double f_code = 1.023e6 + aid;
    double prop = kd2 * e_c;
    prop = u + prop;
    f_code = f_code + prop;

    double xw = f_carr * sfs;
    double xr = f_code * sfs;
    if (xw > 9.0e18) xw = 9.0e18;
    if (xw < -9.0e18) xw = -9.0e18;
    if (!(xr > 0.0)) xr = 0.0;
    if (xr > 4294967295.0) xr = 4294967295.0;
    ch->w = (int32_t)(uint32_t)(uint64_t)(int64_t)nearbyint(xw);
    ch->r = (uint64_t)nearbyint(xr);
    ch->f_carr = f_carr;
    ch->f_code = f_code;

    /* health window */
    double ip2 = ip * ip;
    double qp2 = qp * qp;
    double pw = ip2 + qp2;
    double df2 = ip2 - qp2;
    ex->sum_abs_ip = ex->sum_abs_ip + fabs(ip);
    ex->sum_power = ex->sum_power + pw;
    ex->sum_diff = ex->sum_diff + df2;
    ex->window_count = ex->window_count + 1;
    if (window > 0 && ex->window_count == window) {
        double K = (double)window;
        double m = ex->sum_abs_ip / K;
        double pd = m * m;
        double pt = ex->sum_power / K;
        double pn = pt - pd;
        double cn0 = 0.0;
        if (pn > 0.0) {
            cn0 = pd / pn;
            cn0 = cn0 * inv_T;
        }
        double lock = 0.0;
        if (ex->sum_power > 0.0) lock = ex->sum_diff / ex->sum_power;
        ex->cn0_hz = cn0;
        ex->lock_ratio = lock;
        if (lock < 0.85) ex->lock_fail = ex->lock_fail + 1;
        ex->sum_abs_ip = 0.0;
        ex->sum_power = 0.0;
        ex->sum_diff = 0.0;
        ex->window_count = 0;
    }
    ex->prev_ip = ipi;
    ex->prev_qp = qpi;
    ex->have_prev = 1;
}

/* ------------------------------------------------------------------------ */
/* A whole receiver: blocks in order, channels independent (Sec. 3.5)       */
/* ------------------------------------------------------------------------ */

/*
 * iq: n_blocks * N complex int8 samples, interleaved I,Q.
 * tap_off: [n_ch][n_taps] 32.32 chip offsets.  Every L blocks each channel
 * dumps its accumulators to dumps[(b+1)/L - 1][ch][tap][2], runs orc_track and
 * clears them.  Returns 0, or -1 on bad arguments.
 */
static int orc_run(const int8_t *iq, uint32_t n_blocks, uint32_t N, double fs,
                   uint32_t n_ch, const uint8_t *prn, uint32_t n_taps,
                   const int64_t *tap_off, uint32_t L, int tap_e, int tap_p,
                   int tap_l, double pll_bn, double dll_bn, double fll_bn,
                   uint32_t window, orc_chan *ch, orc_ext *ex, int32_t *dumps);

int orc_run_receiver(const int8_t *iq, uint32_t n_blocks, uint32_t N, double fs,
                     uint32_t n_ch, const uint8_t *prn, uint32_t n_taps,
                     const int64_t *tap_off, uint32_t L, int tap_e, int tap_p,
                     int tap_l, double pll_bn, double dll_bn, orc_chan *ch,
                     int32_t *dumps) {
    return orc_run(iq, n_blocks, N, fs, n_ch, prn, n_taps, tap_off, L, tap_e, tap_p, tap_l,
                   pll_bn, dll_bn, 0.0, 0, ch, NULL, dumps);
}

/* As orc_run_receiver with Table 3's full loop set (orc_track_table3); ex holds
 * each channel's extra state (in and out). */
int orc_run_receiver_table3(const int8_t *iq, uint32_t n_blocks, uint32_t N, double fs,
                            uint32_t n_ch, const uint8_t *prn, uint32_t n_taps,
                            const int64_t *tap_off, uint32_t L, int tap_e, int tap_p,
                            int tap_l, double pll_bn, double dll_bn, double fll_bn,
                            uint32_t window, orc_chan *ch, orc_ext *ex, int32_t *dumps) {
    if (!ex) return -1;
    return orc_run(iq, n_blocks, N, fs, n_ch, prn, n_taps, tap_off, L, tap_e, tap_p, tap_l,
                   pll_bn, dll_bn, fll_bn, window, ch, ex, dumps);
}

static int orc_run(const int8_t *iq, uint32_t n_blocks, uint32_t N, double fs,
                   uint32_t n_ch, const uint8_t *prn, uint32_t n_taps,
                   const int64_t *tap_off, uint32_t L, int tap_e, int tap_p,
                   int tap_l, double pll_bn, double dll_bn, double fll_bn,
                   uint32_t window, orc_chan *ch, orc_ext *ex, int32_t *dumps) {
    if (L == 0 || n_taps == 0) return -1;
    if (tap_e < 0 || tap_p < 0 || tap_l < 0 || (uint32_t)tap_e >= n_taps ||
        (uint32_t)tap_p >= n_taps || (uint32_t)tap_l >= n_taps)
        return -1;
    int8_t *codes = (int8_t *)malloc((size_t)n_ch * ORC_CODE_LEN);
    int32_t *acc = (int32_t *)calloc((size_t)n_ch * n_taps * 2, sizeof(int32_t));
    if (!codes || !acc) { free(codes); free(acc); return -1; }
    for (uint32_t c = 0; c < n_ch; ++c) {
        if (orc_ca_code(prn[c], codes + (size_t)c * ORC_CODE_LEN) != 0) {
            free(codes); free(acc); return -1;
        }
    }
    for (uint32_t b = 0; b < n_blocks; ++b) {
        const int8_t *blk = iq + (size_t)b * N * 2;
        for (uint32_t c = 0; c < n_ch; ++c) {
            orc_correlate_block(blk, N, &ch[c].theta, ch[c].w, &ch[c].phi, ch[c].r,
                                tap_off + (size_t)c * n_taps, n_taps,
                                codes + (size_t)c * ORC_CODE_LEN,
                                acc + (size_t)c * n_taps * 2);
        }
        if ((b + 1) % L == 0) {
            size_t e = (b + 1) / L - 1;
            for (uint32_t c = 0; c < n_ch; ++c) {
                int32_t *a = acc + (size_t)c * n_taps * 2;
                memcpy(dumps + ((e * n_ch + c) * n_taps) * 2, a,
                       sizeof(int32_t) * n_taps * 2);
                if (ex)
                    orc_track_table3(&ch[c], &ex[c], a, tap_off + (size_t)c * n_taps, tap_e,
                                     tap_p, tap_l, fs, (uint64_t)L * N, pll_bn, dll_bn, fll_bn,
                                     window);
                else
                    orc_track(&ch[c], a, tap_off + (size_t)c * n_taps, tap_e, tap_p,
                              tap_l, fs, (uint64_t)L * N, pll_bn, dll_bn);
                memset(a, 0, sizeof(int32_t) * n_taps * 2);
            }
        }
    }
    free(codes);
    free(acc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Acquisition search (Sec. 3.3 ACQ module, Sec. 3.6 outputs, Sec. 3.7)     */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t peak;       /* S at the best cell */
    uint64_t second;     /* best S in the best cell's Doppler row, more than a chip away */
    uint32_t dopp_bin;   /* Doppler bin of the best cell */
    uint32_t code_phase; /* code delay of the best cell, samples, 0..N-1 */
} orc_acq_result;

/*
 * Search one PRN over n_dopp Doppler bins (carrier words w[d]) and every code
 * delay of an acquisition buffer of n_ms blocks of N samples: the ACQ
 * module's buffer of Sec. 3.3, filled for the configured integration length,
 * and the outputs of Sec. 3.6 (PRN, acquisition ratio, coarse Doppler, code
 * delay).  The parallel-code-phase search of Sec. 3.7 evaluates with FFTs the
 * circular correlation of each carrier-wiped block with the local code at all
 * delays at once; here that correlation is written out by its definition, one
 * delay at a time:
 *
 *   g[k]   = code[((k r0) mod 1023*2^32) >> 32],  k = 0..N-1
 *            (the local code sampled from phase 0 with code rate word r0)
 *   theta  = (m N + k) w[d]                       (mod 2^32, 0 at the buffer start)
 *   (c, s) = TAB[theta >> 26]
 *   I'[k]  = I c + Q s,  Q'[k] = Q c - I s        (sample m N + k; exp(-j theta))
 *   Z_I(c) = sum_k I'[k] g[(k - c) mod N],  Z_Q(c) likewise      (exact)
 *   S[d][c] = sum over blocks m of Z_I(c)^2 + Z_Q(c)^2             (mod 2^64)
 *
 * c is the delay of the local code in samples.  The best cell is the largest
 * S, the first in (d, c) order among equals.  With E = ceil(N / 1023) samples
 * (one chip), second is the largest S[d_best][c] over delays whose circular
 * distance min(|c - c_best|, N - |c - c_best|) exceeds E, or 0 if none does.
 * grid, when not NULL, receives S as [n_dopp][N].  Returns 0, or -1 on bad
 * arguments.
 */
int orc_acquire(const int8_t *iq, uint32_t N, uint32_t n_ms, int prn, uint32_t n_dopp,
                const int32_t *w, uint64_t r0, uint64_t *grid, orc_acq_result *out) {
    if (N == 0 || n_ms == 0 || n_dopp == 0 || !iq || !w || !out) return -1;
    int8_t code[ORC_CODE_LEN];
    if (orc_ca_code(prn, code) != 0) return -1;
    int8_t ctab[64], stab[64];
    orc_sincos_table(ctab, stab);

    int8_t *g = (int8_t *)malloc(N);
    int64_t *Ip = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *Qp = (int64_t *)malloc(sizeof(int64_t) * N);
    uint64_t *S = grid ? grid : (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n_dopp * N);
    if (!g || !Ip || !Qp || !S) {
        free(g); free(Ip); free(Qp);
        if (!grid) free(S);
        return -1;
    }
    for (uint32_t k = 0; k < N; ++k) {
        uint64_t ph = (uint64_t)(((unsigned __int128)k * r0) % ORC_CODE_MOD);
        g[k] = code[ph >> 32];
    }
    memset(S, 0, sizeof(uint64_t) * (size_t)n_dopp * N);

    for (uint32_t d = 0; d < n_dopp; ++d) {
        for (uint32_t m = 0; m < n_ms; ++m) {
            const int8_t *blk = iq + (size_t)m * N * 2;
            for (uint32_t k = 0; k < N; ++k) {
                uint32_t n = m * N + k;                     /* sample index, mod 2^32 */
                uint32_t theta = n * (uint32_t)w[d];
                uint32_t t = theta >> 26;
                int64_t c = ctab[t], s = stab[t];
                int64_t I = blk[2 * (size_t)k], Q = blk[2 * (size_t)k + 1];
                Ip[k] = I * c + Q * s;
                Qp[k] = Q * c - I * s;
            }
            for (uint32_t c = 0; c < N; ++c) {
                int64_t zi = 0, zq = 0;
                for (uint32_t k = 0; k < N; ++k) {
                    uint32_t j = k >= c ? k - c : k + N - c;
                    zi += Ip[k] * g[j];
                    zq += Qp[k] * g[j];
                }
                S[(size_t)d * N + c] += (uint64_t)(zi * zi) + (uint64_t)(zq * zq);
            }
        }
    }

    uint64_t best = S[0];
    uint32_t bd = 0, bc = 0;
    for (uint32_t d = 0; d < n_dopp; ++d)
        for (uint32_t c = 0; c < N; ++c)
            if (S[(size_t)d * N + c] > best) {
                best = S[(size_t)d * N + c];
                bd = d;
                bc = c;
            }
    uint32_t E = (N + ORC_CODE_LEN - 1) / ORC_CODE_LEN;
    uint64_t second = 0;
    for (uint32_t c = 0; c < N; ++c) {
        uint32_t dist = c > bc ? c - bc : bc - c;
        if (N - dist < dist) dist = N - dist;
        if (dist > E && S[(size_t)bd * N + c] > second) second = S[(size_t)bd * N + c];
    }
    out->peak = best;
    out->second = second;
    out->dopp_bin = bd;
    out->code_phase = bc;

    free(g); free(Ip); free(Qp);
    if (!grid) free(S);
    return 0;
}

/*
 * Starting NCO words of a tracking channel from an acquisition result (the
 * hand-over from ACQ to tracking of Sec. 3.3).  The local code delayed by c
 * samples matched the received code, so the received code phase at buffer
 * sample 0 is ((N - c) mod N) r0; it advances at the handed-over rate r for
 * the n_ms N samples of the buffer.  The carrier word is the bin's; the code
 * rate is carrier aided as in the loop update of orc_track:
 *   f = w fs / 2^32;  f_code = 1.023e6 + f / 1540;  r = rn(f_code 2^32 / fs)
 *   phi = ((N - c) mod N) r0 + n_ms N r               (mod 1023*2^32)
 * phi is the code phase at the first sample after the buffer.
 */
void orc_acq_handoff(int32_t w, uint32_t code_phase, uint32_t N, uint32_t n_ms, uint64_t r0,
                     double fs, uint64_t *phi, uint64_t *r) {
    double f = (double)w * fs;
    f = f / 4294967296.0;
    double aid = f * ORC_KAID;
    double f_code = 1.023e6 + aid;
    double sfs = 4294967296.0 / fs;
    double xr = f_code * sfs;
    if (!(xr > 0.0)) xr = 0.0;
    if (xr > 4294967295.0) xr = 4294967295.0;
    *r = (uint64_t)nearbyint(xr);
    uint32_t lag = code_phase % N;
    lag = lag == 0 ? 0 : N - lag;
    unsigned __int128 p = (unsigned __int128)lag * r0 + (unsigned __int128)n_ms * N * (*r);
    *phi = (uint64_t)(p % ORC_CODE_MOD);
}

/* ------------------------------------------------------------------------ */
/* Code-period epochs and bit synchronisation (Sec. 3.1, Fig. 7, Sec. 3.6)  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t last_ip;          /* prompt I of the previous epoch */
    uint32_t have_last;
    uint32_t hist[20];        /* sign changes by epoch index mod 20 */
    uint32_t n_changes;
    uint32_t epoch;           /* epochs seen so far (index of the next one) */
    uint32_t sync;            /* 1 once the bit edge is found */
    uint32_t edge;            /* epoch index mod 20 at which a bit starts */
    uint32_t bit_active;      /* 1 while a bit is being integrated */
    uint32_t n_bits;          /* bits decoded */
    int64_t bit_acc;          /* prompt I summed over the current bit's epochs */
    uint64_t bits;            /* the last 64 decoded bits, newest in bit 0 (1 = negative sum) */
    uint32_t first_bit_epoch; /* epoch index at which the first decoded bit starts */
    uint32_t pad;
} orc_bitsync;

/*
 * Bit synchronisation by a histogram of prompt sign changes.  A data bit lasts
 * 20 code periods (Sec. 3.1), so data transitions fall only on every 20th
 * code epoch.  Called once per closed one-period epoch with its prompt I:
 *   - a change of sign from the previous epoch (negative = below zero) counts
 *     in bin (epoch index mod 20);
 *   - before synchronisation: when the fullest bin m (the first among equals)
 *     holds at least k changes and at least 3 times as many as any other bin,
 *     the bit edge is m;
 *   - after it: the prompt I is summed over each bit, from an epoch with index
 *     = edge (mod 20) to the next; at that next epoch the sum's sign is the
 *     decoded bit (1 for a negative sum), shifted into `bits`.
 */
void orc_bitsync_update(orc_bitsync *b, int32_t ip, uint32_t k) {
    uint32_t e = b->epoch;
    uint32_t bin = e % 20;
    if (b->have_last && ((ip < 0) != (b->last_ip < 0))) {
        b->hist[bin] += 1;
        b->n_changes += 1;
    }
    b->last_ip = ip;
    b->have_last = 1;
    if (b->sync) {
        if (bin == b->edge) {
            if (b->bit_active) {
                b->bits = (b->bits << 1) | (uint64_t)(b->bit_acc < 0 ? 1 : 0);
                b->n_bits += 1;
            } else {
                b->first_bit_epoch = e;
            }
            b->bit_active = 1;
            b->bit_acc = 0;
        }
        if (b->bit_active) b->bit_acc += ip;
    } else {
        uint32_t m = 0;
        for (uint32_t j = 1; j < 20; ++j)
            if (b->hist[j] > b->hist[m]) m = j;
        uint32_t second = 0;
        for (uint32_t j = 0; j < 20; ++j)
            if (j != m && b->hist[j] > second) second = b->hist[j];
        if (b->hist[m] >= k && b->hist[m] >= 3 * second) {
            b->sync = 1;
            b->edge = m;
        }
    }
    b->epoch = e + 1;
}

/*
 * Tracking of one channel in code-period epochs, the classic receiver's
 * integrate-and-dump (one code period, Sec. 3.1 / Fig. 7), instead of the
 * fixed sample blocks of orc_run_receiver.  The samples are correlated with
 * the definition of orc_correlate_block.  An epoch ends after the sample at
 * which the prompt code phase, advanced by r, reaches the end of the period:
 * from phase phi that is b = ceil((1023*2^32 - phi) / r) samples.  At the end
 * the accumulators are dumped with the epoch's sample count n, the loops of
 * orc_track run with n_accum = n (T = n / fs), the bit synchroniser gets the
 * prompt I, and the accumulators clear.  acc ([n_taps][2]) and *n_in (samples
 * so far in the open epoch) carry a partial epoch from call to call.  Up to
 * max_epochs closed epochs go to dumps ([max_epochs][n_taps][2]) and
 * epoch_len.  Returns the number of epochs closed, -1 on bad arguments, -2 if
 * more than max_epochs closed.
 */
int orc_track_code_channel(const int8_t *iq, uint64_t nsamp, double fs, int prn,
                           uint32_t n_taps, const int64_t *tap_off, int tap_e, int tap_p,
                           int tap_l, double pll_bn, double dll_bn, uint32_t sync_k,
                           orc_chan *ch, orc_bitsync *bs, int32_t *acc, uint32_t *n_in,
                           uint32_t max_epochs, int32_t *dumps, uint32_t *epoch_len) {
    int8_t code[ORC_CODE_LEN];
    if (orc_ca_code(prn, code) != 0 || n_taps == 0) return -1;
    if (tap_e < 0 || tap_p < 0 || tap_l < 0 || (uint32_t)tap_e >= n_taps ||
        (uint32_t)tap_p >= n_taps || (uint32_t)tap_l >= n_taps)
        return -1;
    uint32_t closed = 0;
    uint64_t pos = 0;
    while (pos < nsamp) {
        uint64_t left = nsamp - pos;
        uint64_t b = UINT64_MAX;                     /* samples to the end of the period */
        if (ch->r != 0) b = (ORC_CODE_MOD - ch->phi + ch->r - 1) / ch->r;
        uint64_t seg = b < left ? b : left;
        orc_correlate_block(iq + 2 * pos, (uint32_t)seg, &ch->theta, ch->w, &ch->phi, ch->r, tap_off,
                            n_taps, code, acc);
        *n_in += (uint32_t)seg;
        pos += seg;
        if (seg == b) {
            if (closed >= max_epochs) return -2;
            memcpy(dumps + (size_t)closed * n_taps * 2, acc, sizeof(int32_t) * n_taps * 2);
            epoch_len[closed] = *n_in;
            orc_track(ch, acc, tap_off, tap_e, tap_p, tap_l, fs, *n_in, pll_bn, dll_bn);
            orc_bitsync_update(bs, acc[2 * tap_p], sync_k);
            memset(acc, 0, sizeof(int32_t) * n_taps * 2);
            *n_in = 0;
            closed += 1;
        }
    }
    return (int)closed;
}
